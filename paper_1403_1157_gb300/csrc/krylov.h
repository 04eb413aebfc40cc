// Launchers of the Krylov vector kernels (krylov.cu).
#pragma once

#include <cuda_runtime.h>

namespace cdg2 {

constexpr int MAX_KRYLOV = 64;   // largest GMRES restart length

// Coefficients passed by value to a kernel (at most MAX_KRYLOV + 1).
struct Coeffs {
    double v[MAX_KRYLOV + 1];
};

template <typename T>
cudaError_t vec_axpby(long long n, double a, const T* x, double b, T* y, cudaStream_t st);
cudaError_t vec_lincomb(long long n, const double* x, int nv, const double* V, long long ldv, const Coeffs& c,
                        double* out, cudaStream_t st);
cudaError_t vec_newton_residual(long long n, const double* Y, const double* fY, double gdt, const double* rhs,
                                double* G, cudaStream_t st);
template <typename S, typename D>
cudaError_t vec_convert(long long n, const S* src, double scale, D* dst, cudaStream_t st);
template <typename T>
cudaError_t vec_add_into(long long n, const T* x, double* y, cudaStream_t st);
// out[j] = V_j . w for j < nv (V_j = V + j * ldv); part: reduction_scratch_doubles(nv) doubles
template <typename T>
cudaError_t vec_mdot(long long n, int nv, const T* V, long long ldv, const T* w, double* part, double* out,
                     cudaStream_t st);
// as vec_mdot, and out[nv] = w . w (the norm before projection) in the same pass
template <typename T>
cudaError_t vec_mdot_self(long long n, int nv, const T* V, long long ldv, const T* w, double* part, double* out,
                          cudaStream_t st);
// w -= sum_j h_j V_j and *norm2_out = |w|^2 after the update, in one pass
template <typename T>
cudaError_t vec_update_norm(long long n, int nv, const T* V, long long ldv, const double* h, T* w, double* part,
                            double* norm2_out, cudaStream_t st);
// True when the 16-byte (packed) kernels below apply: n and ldv multiples of
// 16 / sizeof(T) and both base pointers 16-byte aligned.
template <typename T>
bool vec_packed(long long n, const void* V, long long ldv, const void* w);
// The dot pass of one Arnoldi step with nv = j + 1 basis vectors (packed
// layout): dots[0..nv) = V^T w, dots[nv..2nv) = V^T V_j, dots[2nv] = w . w;
// then column j of the Gram matrix G (ldg x ldg, device) and the CGS2
// coefficients h = 2 V^T w - G V^T w (device, nv doubles).  part:
// reduction_scratch_doubles(2 nv + 1) doubles.
template <typename T>
cudaError_t vec_gs_dots(long long n, int nv, const T* V, long long ldv, const T* w, double* part, double* dots,
                        double* G, int ldg, double* h, cudaStream_t st);
// vec_update_norm over 16-byte packs (packed layout)
template <typename T>
cudaError_t vec_update_norm16(long long n, int nv, const T* V, long long ldv, const double* h, T* w, double* part,
                              double* norm2_out, cudaStream_t st);
template <typename T>
cudaError_t vec_basis_combine(long long n, int nv, const T* V, long long ldv, const Coeffs& y, T* x,
                              cudaStream_t st);
template <typename T>
cudaError_t vec_scale_modes(long long n, const double* table, int period, T* x, cudaStream_t st);
long long reduction_scratch_doubles(int max_vectors);

}  // namespace cdg2
