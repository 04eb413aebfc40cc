"""Two host threads on one device, each with its own mesh and stream.

The one-time set-up of the kernels (their opt-in shared-memory sizes) is done
once per device and must be safe when two threads reach it together; each
mesh owns its workspaces, so the threads share nothing else.  Both threads'
results must equal the single-threaded ones bit for bit.
"""
import threading

import pytest
import torch

import cdg2_inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import paper_1403_1157_gb300 as G
    from paper_1403_1157_gb300 import build
    build.build()
    return G


CASES = [(2, (24, 8), 3), (3, (6, 4, 4), 3), (3, (8, 4, 4), 2)]


def _run(G, dim, cells, k, flags, seed):
    ext, per = (1.0, 0.2, 0.2), ((1, 0, 0) if dim == 2 else (1, 0, 1))
    mesh = G.cdg2_mesh_create(dim, cells, ext, per, k)
    p = I.default_params()
    dt = torch.float32 if flags & G.CDG2_FP32 else torch.float64
    U = torch.from_numpy(I.random_coefficients(mesh.n_elem, mesh.n_basis, seed)).reshape(-1).to("cuda", dt)
    dU = torch.from_numpy(I.random_coefficients(mesh.n_elem, mesh.n_basis, seed + 1)).reshape(-1).to("cuda", dt)
    out_a, out_j, out_v = torch.empty_like(U), torch.empty_like(U), torch.empty_like(U)
    gth = torch.zeros(8, dtype=torch.float64, device="cuda")
    G.cdg2_apply(mesh, p, U, out_a, flags)
    G.cdg2_jvp(mesh, p, U, dU, out_j, flags)
    G.cdg2_vjp(mesh, p, U, dU, out_v, gth, flags)
    torch.cuda.current_stream().synchronize()
    return out_a.cpu(), out_j.cpu(), out_v.cpu(), gth.cpu()


def test_two_threads_one_device(G):
    jobs = [(c, f, 3 + i) for i, c in enumerate(CASES) for f in (G.CDG2_MINV, G.CDG2_MINV | G.CDG2_FP32)]
    want = [_run(G, *c, f, s) for c, f, s in jobs]
    got = [None] * len(jobs)
    errors = []

    def worker(idx):
        try:
            with torch.cuda.stream(torch.cuda.Stream()):
                for j in idx:
                    c, f, s = jobs[j]
                    got[j] = _run(G, *c, f, s)
        except Exception as exc:   # reported below, on the main thread
            errors.append(exc)

    threads = [threading.Thread(target=worker, args=(list(range(w, len(jobs), 2)),)) for w in range(2)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert not errors, errors
    for w, g in zip(want, got):
        for a, b in zip(w, g):
            assert torch.equal(a, b)
