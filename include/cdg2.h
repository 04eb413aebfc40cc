/*
 * cdg2.h -- C ABI of the GB300 CDG2 library for the six-species
 * atherosclerosis model of Girke, Kloefkorn and Ohlberger (arXiv 1403.1157).
 *
 * The library applies the discontinuous Galerkin spatial operator
 *   f(U) = M^{-1} L_h(U),     <phi, L_h(U)> = <phi, K_h(U)> + <phi, I_h(U)>
 * (Sec. 3.1 Eq. convDiscr with the element integrals of Eq. elementint and the
 * surface integrals of Eq. surfaceint; Sec. 3.2 Eq. ode for M^{-1}), its
 * derivatives, and SDIRK time steps solved by Jacobian-free Newton-GMRES
 * (Sec. 3.2).  Every entry point runs its arithmetic in hand-written CUDA
 * kernels for sm_103a on the caller's stream.
 *
 * Conventions shared by all entry points
 * --------------------------------------
 * Mesh: uniform Cartesian cells of the box [0,L0]x[0,L1](x[0,L2]), numbered
 *   lexicographically with x fastest.  Axis 1 (y) is the wall: y = 0 is
 *   Gamma_1 (lumen side), y = L1 is Gamma_2 (outer wall) unless periodic.
 * Basis: on each cell the tensor Legendre basis
 *   phi_i(x) = prod_j sqrt(2 a_j + 1) P_{a_j}(2 xi_j - 1),  xi = (x - x_K)/h,
 *   degree k in each direction (Q_k), multi-index a lexicographic, x fastest;
 *   orthonormal on the unit cell, so M_K = |K| I.
 * Coefficients: U[e][s][i], e < n_elem, s < 6 in the species order
 *   (n1, n2, n3, c1, c2, c3), i < n_basis = (k+1)^dim; contiguous.
 *   float64, or float32 with CDG2_FP32.
 * Pointers: "device" arrays live in GPU memory owned by the caller; the
 *   library never frees them.  Host structs are read during the call only.
 * stream: a cudaStream_t passed as void* (NULL = legacy default stream).
 *   Calls are asynchronous with respect to the host unless stated.
 * Errors: every int-returning call returns CDG2_OK (0) or a negative code;
 *   cdg2_last_error() then describes it.  No call aborts or throws.
 * Domain: the tactic sensitivities chi0 x / (y + chith) of Sec. 2 have a pole
 *   at y = -chith.  Every kernel that evaluates them records, in a status
 *   word of the mesh, whether some quadrature point had y + chith <= 0 (a
 *   test on the sign bits; no trap, no abort).  The operator entry points
 *   (cdg2_apply, cdg2_jvp, cdg2_vjp and their triangle / tetrahedral
 *   counterparts) then wait for their kernels and return CDG2_ERR_DOMAIN if
 *   the word is set (out is then undefined), clearing it.  With CDG2_ASYNC
 *   in flags they return as soon as the work is queued and leave the word
 *   set; the next call without CDG2_ASYNC on the mesh, or
 *   cdg2_mesh_status(), reports it.  The steps check the converged stage
 *   values: a stage value with y + chith <= 0 at a quadrature point returns
 *   CDG2_ERR_DOMAIN (U unchanged), while Newton may pass through iterates
 *   outside the domain on the way; the adjoint step reports stage values
 *   outside it.  The steps leave the word clear.  The status
 *   word (one int of device memory) is allocated by the first call on the
 *   mesh that launches a kernel.
 */
#ifndef CDG2_H
#define CDG2_H

#ifdef __cplusplus
extern "C" {
#endif

#define CDG2_OK 0
#define CDG2_ERR_INVALID_ARG (-1)   /* a NULL pointer, bad size or unsupported option */
#define CDG2_ERR_CUDA (-2)          /* a CUDA runtime call or kernel launch failed */
#define CDG2_ERR_NOT_CONVERGED (-3) /* Newton or GMRES hit its iteration cap */
#define CDG2_ERR_NONFINITE (-4)     /* a NaN or Inf appeared in a solver residual */
#define CDG2_ERR_DOMAIN (-5)        /* c + chi^th <= 0 at a quadrature point: the pole of
                                       chi(x, y, a, b) = a x / (y + b) (Sec. 2) */

/* flags of cdg2_apply / cdg2_jvp / cdg2_vjp */
#define CDG2_MINV 1      /* return M^{-1} L_h (else the residual <phi, L_h>) */
#define CDG2_FORCING 2   /* add the manufactured-solution forcing at time t */
#define CDG2_FP32 4      /* arrays are float32 and the kernel computes in FP32 */
#define CDG2_ASYNC 8     /* do not wait for the domain check (see "Domain" below) */
#define CDG2_TF32 16     /* with CDG2_FP32 on 3D Q3 meshes (apply, JVP): the element
                            contractions on the tensor cores in TF32 (FP32 accumulation) */

/* diffusion fluxes of cdg2_mesh_desc.flux */
#define CDG2_FLUX_CDG2 0
#define CDG2_FLUX_BR2 1
#define CDG2_FLUX_SIPG 2

/* time-stepping schemes of cdg2_step */
#define CDG2_SDIRK2 2    /* Alexander's 2-stage L-stable SDIRK, order 2 */
#define CDG2_SDIRK3 3    /* Alexander's 3-stage L-stable SDIRK, order 3 */
#define CDG2_SDIRK4 4    /* Hairer and Wanner's 5-stage L-stable SDIRK, gamma = 1/4, order 4 */

typedef struct cdg2_mesh cdg2_mesh;

/* Mesh description.
 * dim: 2 or 3.  cells[d] >= 1, extent[d] > 0, periodic[d] in {0,1} for d < dim.
 * k: polynomial degree 1..3 (Q_k, Sec. 3.1 "P_k(K)" read as Q_k on boxes).
 * q1: Gauss points per direction; 0 selects k+2 (the only supported value).
 * chi_e: CDG2 lifting factor (Sec. 3.1: half the faces per element);
 *   <= 0 selects dim (2 for quads, 3 for hexes).
 * gamma1_in: x-range [x0, x1] of the LDL inflow part Gamma_{1,in} of Gamma_1.
 * flux: diffusion flux A^ of Eq. (surfaceint): CDG2_FLUX_CDG2 (0, the paper's
 *   choice), CDG2_FLUX_BR2 (1: eta {A r_e([U])}, liftings on both cells) or
 *   CDG2_FLUX_SIPG (2: interior penalty -C (k+1)^2 A [U] / h) -- the schemes
 *   compared in Fig. 2.  penalty: eta of BR2 (<= 0: 2 dim, the number of
 *   faces) or C of SIPG (<= 0: 2 dim); unused for CDG2.  On these uniform
 *   cells all three reduce to a penalty -c (k+1)^2 A Delta / h_a with
 *   c = chi_e (CDG2), eta / 2 (BR2), C (SIPG). */
typedef struct cdg2_mesh_desc {
    int dim;
    int cells[3];
    double extent[3];
    int periodic[3];
    int k;
    int q1;
    double chi_e;
    double gamma1_in[2];
    int flux;
    double penalty;
} cdg2_mesh_desc;

/* Model coefficients of Eq. (1) and Eq. (3) (Sec. 2).
 * mu, nu: motilities (A = diag(mu1,mu2,mu3,nu1,nu2,nu3)).
 * chi0/chith: tactic sensitivities chi(x,y,a,b) = a x / (y + b) with
 *   (a, b) = (chi0[j], chith[j]) for j = 0: n1 up c1, 1: n1 up c3,
 *   2: n2 up c1, 3: n2 down n1.
 * d1, d2 death rates; gamma = F < 0 the debris term; alpha1, alpha2
 *   neutralisation; f1 the (constant) debris production; k_ox oxidation.
 * beta1, beta2, sigma inflow rates; c1_star, c1_star2 thresholds c1*, c1**.
 * bc_sign: +1 reads the normal of Eq. (3) as inward (influx), -1 outward.
 * mms_phase: phases of the manufactured solution used by CDG2_FORCING,
 *   U*_s = 1 + cos(2 pi x + mms_phase[s]) cos(pi y / L1) exp(-t) / 2.
 * model: 0 = the six-species system of Eq. (1); 1 = the reduced model of
 *   Eq. (2) (Sec. 4.2): only n1, n3, c1 evolve; n2, c2, c3 are inactive and
 *   must be zero fields (their rows of f are zero); n1 has no c3-taxis and no
 *   death term, n3 keeps d1 n1 - gamma n1, c1 has no alpha2 term, and only
 *   the n1 inflow of Eq. (3) remains.  Other values are read as 0. */
typedef struct cdg2_params {
    double mu[3];
    double nu[3];
    double chi0[4];
    double chith[4];
    double d1, d2, gamma, alpha1, alpha2, f1, k_ox;
    double beta1, beta2, sigma, c1_star, c1_star2;
    double bc_sign;
    double mms_phase[6];
    int model;
} cdg2_params;

/* Options of cdg2_step.
 * scheme: CDG2_SDIRK2, CDG2_SDIRK3 or CDG2_SDIRK4 (Sec. 3.2 names DIRK of
 *   order 2, 3 or 4 without tableaux; Reading: L-stable stiffly accurate
 *   SDIRK methods of Alexander (orders 2, 3) and Hairer-Wanner (order 4)).
 * mixed: 0 = FP64 Krylov vectors and FP64 JVP; 1 = FP32 Krylov vectors, FP32
 *   JVP about an FP32 copy of the stage iterate, FP64 Newton residual and
 *   update (iterative refinement); 2 = as 1 with the JVP's element
 *   contractions on the tensor cores in TF32 (CDG2_TF32; 3D Q3 meshes only).
 *   The adjoint step treats 2 as 1.
 * flags: 0 or CDG2_FORCING (manufactured-solution forcing at stage times).
 * Newton stops when ||G||_2 <= max(newton_rtol ||G(Y^0)||_2, newton_atol),
 *   G(Y) = Y - dt a_ii f(Y) - rhs_i, Y^0 the previous stage value (U_n first);
 *   at most max_newton corrections per stage.
 * GMRES(gmres_restart) (Arnoldi by classical Gram-Schmidt applied twice,
 *   CGS2, in two passes over the basis: one pass forms V^T w and the new
 *   column of the basis' Gram matrix G, one pass subtracts V (2I - G) V^T w,
 *   which equals the second classical pass in exact arithmetic; a third,
 *   plain pass when |w| falls below 1e-2 of its size; on vector layouts that
 *   the 16-byte kernels cannot take, one classical pass and a second when the
 *   DGKS criterion |w'| < |w|/sqrt(2) flags cancellation) stops at
 *   ||r||_2 <= gmres_rtol ||G||_2 or
 *   after max_gmres iterations per Newton correction; 1 <= gmres_restart <= 64.
 * precond: 0 = none; 1 = right preconditioning by the modal diagonal
 *   P = 1 - dt a_ii A_s d_i of the diffusion part (for an orthonormal mode on
 *   a Cartesian cell the volume and consistency terms cancel on the
 *   diagonal, leaving the CDG2 penalty: d_i = -chi_e (k+1)^2 sum_j
 *   (psi_{a_j}(0)^2 + psi_{a_j}(1)^2) / h_j^2), applied inside the JVP;
 *   2 = element-block Jacobi: P = the (element, species) diagonal blocks
 *   I - dt a_ii A_s K_e of the diffusion part (cdg2_element_block), inverted
 *   on the host once per call (a few distinct blocks per mesh) and applied
 *   by a kernel before every JVP/VJP.  The preconditioner changes the
 *   iteration count, not the converged result.  The adjoint uses the same
 *   P (K_e is symmetric).
 * jacobian: 0 = matrix-free (the JVP kernel in every Krylov iteration);
 *   1 = assembled: before every Newton correction the Jacobian at the
 *   current iterate is assembled (cdg2_assemble_jacobian) and GMRES applies
 *   it with cdg2_spmv; FP64 only (mixed = 0), Cartesian meshes whose
 *   periodic axes have at least 3 cells.  The adjoint step ignores it. */
typedef struct cdg2_solver_opts {
    int scheme;
    int mixed;
    int flags;
    int max_newton;
    int gmres_restart;
    int max_gmres;
    double newton_rtol;
    double newton_atol;
    double gmres_rtol;
    int precond;
    int jacobian;
} cdg2_solver_opts;

/* Statistics of one cdg2_step call. */
typedef struct cdg2_stats {
    int stages;           /* stages of the scheme */
    int newton_iters;     /* Newton corrections, all stages */
    int gmres_iters;      /* GMRES iterations (JVP launches in Arnoldi), all stages */
    double residual0[5];  /* ||G(Y^0)||_2 per stage */
    double residual[5];   /* final ||G||_2 per stage */
    double seconds;       /* host wall time of the call */
    int gmres_reorth;     /* Arnoldi steps that needed an extra Gram-Schmidt pass */
} cdg2_stats;

/* Build a mesh (host call, synchronous).  Tabulates the 1D basis and Gauss
 * rule on the host.  *out receives an opaque handle owned by the caller
 * until cdg2_mesh_destroy.  Errors: INVALID_ARG for an unsupported desc. */
int cdg2_mesh_create(const cdg2_mesh_desc* desc, cdg2_mesh** out);

/* Free a mesh and every device workspace it owns (synchronises the device
 * work queued on those buffers).  NULL is ignored. */
void cdg2_mesh_destroy(cdg2_mesh* mesh);

/* Sizes: elements, basis functions per species per element, total DOF
 * (= 6 * n_elem * n_basis).  Any output pointer may be NULL. */
int cdg2_mesh_info(const cdg2_mesh* mesh, long long* n_elem, int* n_basis, long long* n_dof);

/* Wait for `stream` and report the mesh's domain status word (see "Domain"
 * above): CDG2_ERR_DOMAIN if a kernel queued on the mesh since the last
 * report met y + chith <= 0 at a quadrature point (the pole of chi, Sec. 2),
 * else CDG2_OK.  Clears the word.  Meant for calls made with CDG2_ASYNC. */
int cdg2_mesh_status(const cdg2_mesh* mesh, void* stream);

/* out = M^{-1} L_h(U) (flags & CDG2_MINV) or out = <phi, L_h(U)>.
 * Sec. 3.1 Eq. convDiscr: element integrals int_K (F - A grad U):grad phi
 * + S.phi; interior faces: symmetric terms {A grad phi}:[U], consistency
 * {A grad U}:[phi], local Lax-Friedrichs F^ and the CDG2 diffusion flux
 * 2 chi_e A r_e([U]) on K^-_e (the lower-coordinate cell); boundary faces:
 * the influxes of Eq. (3).  Sec. 3.2: M^{-1} of the orthonormal basis.
 * U, out: device arrays [n_elem][6][n_basis] (float64, or float32 with
 * CDG2_FP32); they must not overlap.  t: time of the CDG2_FORCING term.
 * Each face is evaluated once into a per-mesh face buffer that the first
 * cdg2_apply or cdg2_jvp on the mesh allocates (cudaMalloc, about
 * 2*6*(k+1)^(dim-1) doubles per face); calls sharing a mesh must therefore
 * be ordered on one stream.  flags may add CDG2_ASYNC, and on 3D Q3 meshes
 * with CDG2_FP32 also CDG2_TF32: the volume terms' basis-to-quadrature and
 * quadrature-to-basis contractions then run as TF32 GEMMs on the tensor
 * cores (16 elements per thread block, accumulators in tensor memory); the
 * pointwise model, the faces and the modal diffusion stay in FP32.  Meant
 * for the inner Krylov operator of the mixed solver: the JVP along a rough
 * tangent keeps about 5e-5 relative to FP64; on smooth states the apply of
 * n1 and n2 (whose chemotactic fluxes go through the tensor cores; every
 * species' diffusion is applied in FP32 modal form) loses up to about 2e-3
 * to the cancellation of the weak form.  With CDG2_TF32, U and dU must be
 * 16-byte aligned (else CDG2_ERR_CUDA, misaligned address); without it any
 * element-aligned array is accepted (the face kernels then load without
 * bulk copies).  Errors: INVALID_ARG,
 * CUDA, DOMAIN (y + chith <= 0 at a quadrature point; out undefined). */
int cdg2_apply(const cdg2_mesh* mesh, const cdg2_params* params, const void* U, void* out,
               int flags, double t, void* stream);

/* Directional derivative of cdg2_apply (the Jacobian-vector product of the
 * Jacobian-free Newton-Krylov solver, Sec. 3.2):
 *   out = J(U) dU + (d f / d theta) dtheta,   f = M^{-1} L_h (CDG2_MINV) or L_h.
 * Linearised pointwise terms: d|x|/dx = sign(x) with sign(0) = 0, the LLF
 * maximum differentiated on the K^- side at a tie, H' = 0, and the forcing
 * (independent of U) drops out.  theta = (d1, d2, gamma, alpha1, alpha2, f1,
 * k_ox, beta1) (the reaction coefficients of Eq. (1) and the immune-cell
 * inflow rate of Eq. (3)); dtheta is a HOST array of 8 doubles or NULL.
 * U, dU, out: device [n_elem][6][n_basis], float64 or float32 (CDG2_FP32);
 * out must not overlap U or dU.  t is accepted for symmetry and unused.
 * flags may add CDG2_ASYNC.  Errors: INVALID_ARG, CUDA, DOMAIN (at U). */
int cdg2_jvp(const cdg2_mesh* mesh, const cdg2_params* params, const void* U, const void* dU,
             const double* dtheta, void* out, int flags, double t, void* stream);

/* One SDIRK step U_n -> U_{n+1} of U' = f(U, t) = M^{-1} L_h(U) (+ forcing)
 * (Sec. 3.2, Eq. ode), each stage solved by Jacobian-free Newton-Krylov with
 * GMRES (Sec. 3.2) on the GPU; JVPs come from cdg2_jvp's kernel.
 * U: device float64 [n_elem][6][n_basis], overwritten with U_{n+1}.
 * t, dt: time and step (dt > 0).  opts: see cdg2_solver_opts.  stats: may be
 * NULL.  Synchronous: returns after the step has completed on `stream`.
 * The first call allocates a per-mesh workspace (cudaMalloc; 8 state vectors
 * plus gmres_restart + 5 Krylov vectors); calls sharing a mesh must be
 * ordered.  Errors: NOT_CONVERGED (U unchanged, stats filled), NONFINITE
 * (a NaN/Inf residual), DOMAIN (a converged stage value with y + chith <= 0
 * at a quadrature point; U unchanged), INVALID_ARG, CUDA. */
int cdg2_step(const cdg2_mesh* mesh, const cdg2_params* params, double* U, double t, double dt,
              const cdg2_solver_opts* opts, cdg2_stats* stats, void* stream);

/* cdg2_step that also stores the converged stage values Y_1..Y_s, the
 * linearisation points of the step's discrete adjoint.
 * stages: device float64 [s][n_elem][6][n_basis] (s = 2, 3, 5 for SDIRK2, 3, 4). */
int cdg2_step_stages(const cdg2_mesh* mesh, const cdg2_params* params, double* U, double t, double dt,
                     const cdg2_solver_opts* opts, double* stages, cdg2_stats* stats, void* stream);

/* Discrete adjoint of one SDIRK step (Sec. 3.2 stepping, differentiated):
 * lam <- (dU_{n+1}/dU_n)^T lam and gtheta += (dU_{n+1}/dtheta)^T lam, theta
 * as in cdg2_jvp.  With K_i = f(Y_i): backwards over the stages,
 *   r_i = dt b_i lam + dt sum_{j>i} a_ji ybar_j,  (I - dt a_ii J(Y_i)^T) g_i = r_i,
 *   ybar_i = J(Y_i)^T g_i,  gtheta += (df/dtheta)(Y_i)^T g_i,  lam_n = lam + sum_i ybar_i.
 * stages: the output of cdg2_step_stages for this step.  Each stage system
 * is solved to ||residual||_2 <= max(newton_rtol ||r_i||_2, newton_atol) by
 * refinement (FP64 residual via cdg2_vjp's kernel; corrections by GMRES in
 * FP64, or FP32 with opts->mixed); max_newton bounds the refinements.
 * lam: device float64, in/out.  gtheta: device float64 [8], accumulated, or
 * NULL.  opts->flags must be 0 (the forcing's coefficient dependence is not
 * differentiated).  Synchronous; workspace as cdg2_step (+ cdg2_vjp's). */
int cdg2_step_adjoint(const cdg2_mesh* mesh, const cdg2_params* params, const double* stages, double t, double dt,
                      const cdg2_solver_opts* opts, double* lam, double* gtheta, cdg2_stats* stats, void* stream);

/* Transpose of cdg2_jvp (vector-Jacobian product, for the adjoint of the
 * implicit steps):
 *   gU = J(U)^T lam,   gtheta = (d f / d theta)^T lam  (when gtheta != NULL),
 * f = M^{-1} L_h (CDG2_MINV) or L_h, theta as in cdg2_jvp, same derivative
 * conventions.  Each element gathers the adjoint contributions of its own
 * volume and faces (no atomics); gtheta is reduced in a fixed order, so the
 * result is bitwise reproducible.  U, lam, gU: device [n_elem][6][n_basis],
 * float64 or float32 (CDG2_FP32; gtheta is float64 either way); gU must not
 * overlap U or lam.  gtheta: DEVICE array of 8 doubles or NULL.  The first
 * call with gtheta allocates a per-mesh workspace (8 doubles per CTA,
 * cudaMalloc); calls sharing a mesh must then be ordered on one stream.
 * flags may add CDG2_ASYNC.  Errors: INVALID_ARG, CUDA, DOMAIN (at U). */
int cdg2_vjp(const cdg2_mesh* mesh, const cdg2_params* params, const void* U, const void* lam, void* gU,
             double* gtheta, int flags, double t, void* stream);

/* cdg2_vjp for callers that cannot allocate device memory (the paper has no
 * counterpart; this is a library-interface addition).  cdg2_vjp cudaMallocs
 * a per-mesh workspace the first time gtheta is requested; a caller whose
 * device memory is wholly managed by its own pool allocator, or whose loop
 * must never incur the implicit device synchronisation of cudaMalloc /
 * cudaFree, cannot accept that.  This entry point computes the same gU and
 * gtheta with its scratch in a fixed 1 MiB device array inside the library
 * (held on every GPU that loads the library until the process exits) and
 * calls no cudaMalloc, cudaFree or other allocating routine.
 * Limit: with gtheta != NULL the mesh may need at most 16384 VJP thread
 * blocks (elements per block: 2D 8/4/4 for k = 1/2/3, 3D 4/2/1; e.g. 16384
 * 3D Q3 elements); larger meshes return CDG2_ERR_INVALID_ARG.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Under CUDA's lazy module loading (the
 * default) that first call is also when the library's module holding the
 * array is loaded on the device and the array takes its device memory;
 * later calls take none.  All calls share the array and nothing in it
 * needs to start at zero (each block overwrites its own slots), but calls
 * that overlap on the GPU race on it: order them on one stream.  The domain
 * check (see "Domain") uses a second static device word of the library, not
 * the mesh's, so the call needs nothing allocated on the mesh either; the
 * call always waits for its kernels and reads it (flags must not hold
 * CDG2_ASYNC).  Arguments, layouts and results are those of cdg2_vjp. */
int cdg2_vjp_noalloc(const cdg2_mesh* mesh, const cdg2_params* params, const void* U, const void* lam, void* gU,
                     double* gtheta, int flags, double t, void* stream);

/* Initial data: out = L2 projection onto V_h of
 *   u0_s(x) = floor_value + sum_b amps[s][b] exp(-|x - centres[s][b]|^2 / (2 sigma^2))
 * (Sec. 3.2: U(0) is the projection of U_0), distances taken as minimum
 * images along periodic axes, with the q1-point Gauss rule of the mesh.
 * centres: host [6][n_gauss][dim], amps: host [6][n_gauss] (read during the
 * call), 0 <= n_gauss <= 16, sigma > 0.  out: device [n_elem][6][n_basis],
 * float64 or float32 (flags = CDG2_FP32). */
int cdg2_project_gaussians(const cdg2_mesh* mesh, int n_gauss, const double* centres, const double* amps,
                           double sigma, double floor_value, void* out, int flags, void* stream);

/* out = L2 projection of the manufactured solution
 *   U*_s = 1 + cos(2 pi x + params->mms_phase[s]) cos(pi y / L1) exp(-t) / 2
 * (a smooth positive field with zero normal derivative on y = 0, L1).
 * out: device [n_elem][6][n_basis], float64 or float32 (CDG2_FP32). */
int cdg2_project_mms(const cdg2_mesh* mesh, const cdg2_params* params, double t, void* out, int flags,
                     void* stream);

/* ---- Assembled Jacobian (Sec. 3.2) -----------------------------------------
 * Sec. 3.2 solves the stage systems matrix-free and sets a "fully assembled
 * approach" aside; this is that alternative, for comparison: the Jacobian
 * J = d(M^{-1} L_h)/dU at a state U, element-block sparse.  Row block e holds
 * b x b blocks (b = 6 n_basis) for e itself and its 2 dim face neighbours
 * (absent on walls), column-major, in device memory owned by the handle:
 * E (2 dim + 1) b^2 doubles (e.g. 6.0 GB for 2D 256x64 Q3, 0.48 GB for 2D
 * 128x32 Q2).  Assembly probes the JVP (cdg2_jvp's kernel, with M^{-1}) with
 * one (species, mode) of all the elements of one colour of a distance-2
 * element colouring at a time: colours x b JVP launches.  The matrix is
 * tied to its mesh (which must outlive it); calls on one matrix must be
 * ordered on one stream. */
typedef struct cdg2_matrix cdg2_matrix;

/* Allocate the blocks, the neighbour table and the colouring (host call,
 * synchronous; device memory as above).  Errors: INVALID_ARG (NULL, a
 * periodic axis with fewer than 3 cells), CUDA (out of device memory). */
int cdg2_matrix_create(const cdg2_mesh* mesh, cdg2_matrix** out);
void cdg2_matrix_destroy(cdg2_matrix* A);
/* Block size b, blocks per row (2 dim + 1), colours of the colouring, device bytes of the blocks. */
int cdg2_matrix_info(const cdg2_matrix* A, int* block_size, int* slots, int* colours, long long* bytes);
/* A = J(U) (U: device float64 [n_elem][6][n_basis]).  Waits for the stream.
 * Errors: INVALID_ARG, CUDA, DOMAIN (U outside the model's domain). */
int cdg2_assemble_jacobian(cdg2_matrix* A, const cdg2_params* params, const double* U, void* stream);
/* y = alpha A x + beta y (device float64 vectors of n_dof, not overlapping);
 * beta = 0 ignores the old y.  One thread block per row element, the blocks
 * read column by column (coalesced).  Errors: INVALID_ARG, CUDA. */
int cdg2_spmv(const cdg2_matrix* A, double alpha, const double* x, double beta, double* y, void* stream);

/* Human-readable description of the last error on this thread. */
/* The block that precond = 2 inverts, for element `elem` and species
 * `species`: I - gdt A_s K_e (row-major n_basis x n_basis, host memory
 * `out`), where K_e is the diagonal block of the diffusion part of
 * M^{-1} L_h (Sec. 3.1 Eq. convDiscr with only the A terms: the volume
 * stiffness and the element's own terms of the consistency, symmetry and
 * penalty (CDG2: chi_e (k+1)^2 / h; BR2, SIPG: their constants) parts of
 * its interior faces; boundary faces add nothing).  The paper defers
 * assembled operators and preconditioners (Sec. 3.2); this block is the
 * one piece of the assembled operator the solver uses.  Host-only (no
 * device work); gdt may be any finite value.  Errors: INVALID_ARG (NULL,
 * elem or species out of range). */
int cdg2_element_block(const cdg2_mesh* mesh, const cdg2_params* params, double gdt, long long elem, int species,
                       double* out);

/* ---- Triangle meshes (Sec. 3.1: P_k on triangles, chi_e = 1.5) ----------
 * The operator f(U) = M^{-1} L_h(U) of cdg2_apply on an affine triangle
 * mesh, FP64.  Readings (the paper fixes none of them): on the reference
 * triangle {xi, eta >= 0, xi + eta <= 1} the orthonormal Dubiner basis
 * psi_pq = sqrt(2 (2p+1) (p+q+1)) (1-eta)^p P_p(2 xi/(1-eta) - 1)
 * P_q^{(2p+1,0)}(2 eta - 1), modes ordered by p + q then q, mapped by
 * x = x_0 + [x_1 - x_0, x_2 - x_0] (xi, eta) (so M_K = 2 |K| I); the
 * collapsed Gauss rule with (k+2)^2 volume points and k+2 points per edge;
 * K^-_e the smaller adjacent triangle (Sec. 3.1; areas within a relative
 * 1e-12 tie, a tie goes to the lower triangle index); boundary edges on
 * y = 0 are Gamma_1 and on y = max y Gamma_2 (Eq. (3)), every other boundary
 * edge is a no-flow wall.  Layout of U and out: [n_tri][6][n_basis],
 * n_basis = (k+1)(k+2)/2. */
typedef struct cdg2_tri_mesh cdg2_tri_mesh;

typedef struct cdg2_tri_desc {
    long long n_vert;
    const double* xy;        /* host [n_vert][2] vertex coordinates */
    long long n_tri;
    const long long* tri;    /* host [n_tri][3] vertex indices, counter-clockwise */
    int k;                   /* 1..3 */
    double chi_e;            /* CDG2 lifting factor; <= 0 selects 1.5 (Sec. 3.1, triangles) */
    double gamma1_in[2];     /* x-range of Gamma_{1,in} on y = 0 */
} cdg2_tri_desc;

/* Build a triangle mesh (host call; the arrays are copied).  Errors:
 * INVALID_ARG for k outside 1..3, an index out of range, a degenerate or
 * clockwise triangle, neighbours with inconsistent orientation, or an edge
 * shared by more than two triangles.  Device memory is allocated by the first
 * cdg2_tri_apply and freed by cdg2_tri_mesh_destroy (calls sharing a mesh
 * must be ordered on one stream). */
int cdg2_tri_mesh_create(const cdg2_tri_desc* desc, cdg2_tri_mesh** out);
void cdg2_tri_mesh_destroy(cdg2_tri_mesh* mesh);
int cdg2_tri_mesh_info(const cdg2_tri_mesh* mesh, long long* n_elem, int* n_basis, long long* n_dof,
                       long long* n_faces);
/* The domain status of a triangle mesh, as cdg2_mesh_status. */
int cdg2_tri_mesh_status(const cdg2_tri_mesh* mesh, void* stream);

/* out = M^{-1} L_h(U) (flags = CDG2_MINV) or <phi, L_h(U)> (flags = 0) on a
 * triangle mesh; U, out: device float64 [n_tri][6][n_basis], not
 * overlapping.  Two kernels: every interior edge once (traces, the CDG2
 * lifting on K^-, the face flux, its test against both sides) into a face
 * buffer, then every element (volume terms, its edges, boundary data,
 * M^{-1}).  flags may add CDG2_ASYNC.  Errors: INVALID_ARG (NULL, overlap,
 * other flags), CUDA, DOMAIN (y + chith <= 0 at a quadrature point). */
int cdg2_tri_apply(const cdg2_tri_mesh* mesh, const cdg2_params* params, const double* U, double* out, int flags,
                   void* stream);

/* out = J(U) dU, the derivative of cdg2_tri_apply along dU (the linearised
 * element and face terms; the lifting is linear; H' = 0, so the boundary data
 * drop out), same layout and flags.  U, dU, out: device float64, out must
 * not overlap U or dU.  Errors as cdg2_tri_apply. */
int cdg2_tri_jvp(const cdg2_tri_mesh* mesh, const cdg2_params* params, const double* U, const double* dU, double* out,
                 int flags, void* stream);

/* gU = J(U)^T lambda for cdg2_tri_apply with the same flags (CDG2_MINV: the
 * transpose of M^{-1} L_h), as a gather: every interior edge once (the
 * cotangents of its flux back through the flux and the K^- lifting, tested
 * against both sides into the face buffer), then every element (its volume
 * terms and its edges); no atomics, bitwise reproducible.  H' = 0: the
 * boundary data add nothing.  U, lam, gU: device float64, gU must not
 * overlap U or lam.  Errors as cdg2_tri_apply. */
int cdg2_tri_vjp(const cdg2_tri_mesh* mesh, const cdg2_params* params, const double* U, const double* lam,
                 double* gU, int flags, void* stream);

/* One SDIRK step U_n -> U_(n+1) of U' = M^{-1} L_h(U) on a triangle mesh
 * (Sec. 3.2: each stage by Newton's method, each correction by restarted
 * GMRES whose matrix-vector product is one cdg2_tri_jvp and one axpby), FP64,
 * in place on U (device float64, n_dof values).  opts as for cdg2_step with
 * mixed = 0, flags = 0 (no forcing) and precond = 0 (none) or 2 (right
 * preconditioning by element-block Jacobi: the diagonal blocks K_(e,s) of the
 * diffusion part, probed with the diffusion JVP under a distance-1 colouring
 * of the elements and cached until the diffusivities change, and the inverses
 * of I - dt a_ii K_(e,s)); the stage times enter no term.  The mesh owns the
 * workspace and the blocks, allocated by the first call and freed by its
 * destroy.  Errors: INVALID_ARG (NULL, options),
 * NOT_CONVERGED / NONFINITE (stats filled, U unchanged; NONFINITE also for a
 * block that is not positive definite), CUDA. */
int cdg2_tri_step(const cdg2_tri_mesh* mesh, const cdg2_params* params, double* U, double dt,
                  const cdg2_solver_opts* opts, cdg2_stats* stats, void* stream);

/* ---- Tetrahedral meshes (Sec. 3.1: P_k on tetrahedra, chi_e = 2) ----------
 * The operator of cdg2_apply on an affine tetrahedral mesh, FP64.  Readings:
 * on the reference tetrahedron the orthonormal Dubiner basis psi_pqr =
 * c_pqr L_p J_q R_r (L_p = s^p P_p((2 xi - s)/s), s = 1 - eta - zeta; J_q =
 * t^q P_q^{(2p+1,0)}((2 eta - t)/t), t = 1 - zeta; R_r = P_r^{(2p+2q+2,0)}
 * (2 zeta - 1); c_pqr = sqrt((2p+1)(2p+2q+2)(2p+2q+2r+3)); modes by total
 * degree, then r, then q), so M_K = 6 |K| I; the collapsed Gauss rule with
 * (k+2)^3 volume points and the collapsed triangle rule with (k+2)^2 points
 * per face in K^-'s parametrisation (local face l: the vertices other than l
 * in increasing local order); K^-_e the smaller tetrahedron (volumes within a
 * relative 1e-12 tie, a tie goes to the lower index); boundary faces on
 * y = 0 are Gamma_1, on y = max y Gamma_2, other boundary faces are walls.
 * U and out: [n_tet][6][n_basis], n_basis = (k+1)(k+2)(k+3)/6. */
typedef struct cdg2_tet_mesh cdg2_tet_mesh;

typedef struct cdg2_tet_desc {
    long long n_vert;
    const double* xyz;       /* host [n_vert][3] vertex coordinates */
    long long n_tet;
    const long long* tet;    /* host [n_tet][4] vertex indices, positively oriented */
    int k;                   /* 1..3 */
    double chi_e;            /* CDG2 lifting factor; <= 0 selects 2 (Sec. 3.1, tetrahedra) */
    double gamma1_in[2];     /* x-range of Gamma_{1,in} on y = 0 */
} cdg2_tet_desc;

/* Build a tetrahedral mesh (host call; the arrays are copied).  Errors:
 * INVALID_ARG for k outside 1..3, an index out of range, a degenerate or
 * negatively oriented tetrahedron, an inconsistent shared face, or a face of
 * more than two tetrahedra.  Device memory is allocated by the first
 * cdg2_tet_apply and freed by cdg2_tet_mesh_destroy. */
int cdg2_tet_mesh_create(const cdg2_tet_desc* desc, cdg2_tet_mesh** out);
void cdg2_tet_mesh_destroy(cdg2_tet_mesh* mesh);
int cdg2_tet_mesh_info(const cdg2_tet_mesh* mesh, long long* n_elem, int* n_basis, long long* n_dof,
                       long long* n_faces);
/* The domain status of a tetrahedral mesh, as cdg2_mesh_status. */
int cdg2_tet_mesh_status(const cdg2_tet_mesh* mesh, void* stream);

/* out = M^{-1} L_h(U) (flags = CDG2_MINV) or <phi, L_h(U)> (flags = 0) on a
 * tetrahedral mesh; U, out: device float64, not overlapping.  A face kernel
 * (every interior face once: traces of both sides at K^-'s face points, the
 * CDG2 lifting on K^-, the face flux, its test against both sides into a face
 * buffer) and an element kernel (volume terms, its faces, boundary data,
 * M^{-1}).  flags may add CDG2_ASYNC.  Errors: INVALID_ARG (NULL, overlap,
 * other flags), CUDA, DOMAIN (y + chith <= 0 at a quadrature point). */
int cdg2_tet_apply(const cdg2_tet_mesh* mesh, const cdg2_params* params, const double* U, double* out, int flags,
                   void* stream);

/* out = J(U) dU, the derivative of cdg2_tet_apply along dU (the linearised
 * element and face terms; the lifting is linear; H' = 0, so the boundary data
 * drop out), same layout and flags.  U, dU, out: device float64, out must
 * not overlap U or dU.  Errors as cdg2_tet_apply. */
int cdg2_tet_jvp(const cdg2_tet_mesh* mesh, const cdg2_params* params, const double* U, const double* dU, double* out,
                 int flags, void* stream);

/* gU = J(U)^T lambda for cdg2_tet_apply with the same flags (CDG2_MINV: the
 * transpose of M^{-1} L_h), as a gather: every interior face once (the
 * cotangents of its flux back through the flux and the K^- lifting, tested
 * against both sides into the face buffer), then every element (its volume
 * terms and its faces); no atomics, bitwise reproducible.  H' = 0: the
 * boundary data add nothing.  U, lam, gU: device float64, gU must not
 * overlap U or lam.  Errors as cdg2_tet_apply. */
int cdg2_tet_vjp(const cdg2_tet_mesh* mesh, const cdg2_params* params, const double* U, const double* lam,
                 double* gU, int flags, void* stream);

/* One SDIRK step U_n -> U_(n+1) of U' = M^{-1} L_h(U) on a tetrahedral mesh
 * (Sec. 3.2: each stage by Newton's method, each correction by restarted
 * GMRES whose matrix-vector product is one cdg2_tet_jvp and one axpby), FP64,
 * in place on U (device float64, n_dof values).  opts as for cdg2_step with
 * mixed = 0, flags = 0 (no forcing) and precond = 0 (none) or 2 (right
 * preconditioning by element-block Jacobi: the diagonal blocks K_(e,s) of the
 * diffusion part, probed with the diffusion JVP under a distance-1 colouring
 * of the elements and cached until the diffusivities change, and the inverses
 * of I - dt a_ii K_(e,s)); the stage times enter no term.  The mesh owns the
 * workspace and the blocks, allocated by the first call and freed by its
 * destroy.  Errors: INVALID_ARG (NULL, options),
 * NOT_CONVERGED / NONFINITE (stats filled, U unchanged; NONFINITE also for a
 * block that is not positive definite), CUDA. */
int cdg2_tet_step(const cdg2_tet_mesh* mesh, const cdg2_params* params, double* U, double dt,
                  const cdg2_solver_opts* opts, cdg2_stats* stats, void* stream);

/* Measured FMA throughput of the current GPU (the paper has no counterpart;
 * a measurement utility for the roofline of the operator kernels, which are
 * bound by the FP64 or FP32 pipes): kind 0 = FP64, 1 = FP32.  Runs an FMA
 * loop of `iters` (>= 8) steps on 8 independent chains in every thread of
 * 8 x (SM count) blocks of 256 threads on `stream`, timed with CUDA events,
 * and writes 2 x FMAs / time in TFLOP/s to the host double *tflops.
 * Synchronous.  Errors: INVALID_ARG, CUDA. */
int cdg2_probe_peak(int kind, int iters, double* tflops, void* stream);

const char* cdg2_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CDG2_H */
