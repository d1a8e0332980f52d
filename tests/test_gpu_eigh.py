"""The batched Hermitian eigensolver behind Eqs. 4-5 (eph_eigh), against the oracle's
eigendecomposition (numpy's LAPACK eigh) and the properties that any valid
eigendecomposition has (residual A V - V diag(w), unitarity of V), which stay meaningful
inside degenerate subspaces where eigenvectors are not unique.

Sizes cover every solver: register-resident warps (n <= 12: FP32 sweeps + FP64
refinement, with the Jacobi polish as fallback; n = 13..16: plain FP64 sweeps), the
CTA-per-matrix preconditioned solver (17 <= n <= ~230) and the plain FP64 CTA solver
(n = 256, whose packed FP32 copy does not fit in shared memory).  Special spectra:
exact multiplicities, near-degenerate pairs (gaps 1e-4 .. 1e-12 of the spread, which the
refinement cannot resolve and hands to the Jacobi polish), the zero matrix, multiples of the
identity, diagonal and rank-one matrices, and scales of 1e-30 and 1e+30."""
import os

import numpy as np
import pytest

import oracle
from paper_2603_10295_gb300 import binding, build_lib, synth

pytestmark = pytest.mark.gpu

SIZES = [1, 2, 3, 5, 6, 8, 9, 11, 12, 13, 16, 17, 24, 33, 64, 120, 180, 231, 256]
TOL = {"fp64": dict(eig=1e-13, res=1e-13, orth=1e-13), "mixed": dict(eig=2e-11, res=1e-8, orth=1e-8)}


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not os.path.exists(binding.LIB_PATH):
        build_lib.build()
    return binding.load_library()


@pytest.fixture(scope="module")
def ctxs():
    wl = synth.make_workload("si_tiny", nk=4, nq=2)
    return {f: binding.Context.from_workload(wl, form=f) for f in ("fp64", "mixed")}


def rand_herm(rng, batch, n, scale=3.0):
    M = rng.normal(size=(batch, n, n)) + 1j * rng.normal(size=(batch, n, n))
    return scale * (M + np.conj(np.swapaxes(M, 1, 2)))


def with_spectrum(rng, spectra):
    """Q diag(d) Q^H with random unitary Q per row of spectra [batch][n]."""
    spectra = np.asarray(spectra, dtype=np.float64)
    batch, n = spectra.shape
    Z = rng.normal(size=(batch, n, n)) + 1j * rng.normal(size=(batch, n, n))
    Q, _ = np.linalg.qr(Z)
    A = np.einsum("bij,bj,bkj->bik", Q, spectra, np.conj(Q))
    return 0.5 * (A + np.conj(np.swapaxes(A, 1, 2)))


def check(ctx, A, form, what):
    w, V = ctx.eigh(A)
    w_ref, _ = oracle.electron_eigen(A)
    scale = np.maximum(np.abs(w_ref).max(-1), 1e-300)  # ||A||_2 per matrix
    tol = TOL[form]
    n = A.shape[-1]
    e_eig = float((np.abs(w - w_ref).max(-1) / scale).max())
    res = np.einsum("bij,bjk->bik", A, V) - V * w[:, None, :]
    e_res = float((np.abs(res).max((-1, -2)) / scale).max())
    e_orth = float(np.abs(np.einsum("bji,bjk->bik", np.conj(V), V) - np.eye(n)).max())
    print(what, form, dict(eig=e_eig, res=e_res, orth=e_orth))
    assert np.all(np.diff(w, axis=-1) >= 0), (what, "not ascending")
    assert e_eig <= tol["eig"] and e_res <= tol["res"] and e_orth <= tol["orth"], (what, form, e_eig, e_res, e_orth)


@pytest.mark.parametrize("form", ["fp64", "mixed"])
@pytest.mark.parametrize("n", SIZES)
def test_random(ctxs, form, n):
    rng = np.random.default_rng(n)
    batch = 257 if n <= 16 else (40 if n <= 64 else 6)
    check(ctxs[form], rand_herm(rng, batch, n), form, f"random n={n}")


@pytest.mark.parametrize("form", ["fp64", "mixed"])
@pytest.mark.parametrize("n", [4, 8, 11, 12, 16, 17, 64, 120])
def test_special_spectra(ctxs, form, n):
    rng = np.random.default_rng(100 + n)
    base = np.sort(rng.uniform(-10.0, 10.0, size=n))
    spread = base[-1] - base[0]
    rows = []
    m = np.array(base)
    m[: min(3, n)] = m[0]                          # a triple (n >= 3)
    rows.append(m)
    for gap in (1e-4, 1e-7, 1e-10, 1e-12):         # near-degenerate pair in the middle
        m = np.array(base)
        h = n // 2
        m[h] = m[h - 1] + gap * spread
        rows.append(np.sort(m))
    rows.append(np.full(n, 2.5))                   # multiple of the identity
    rows.append(np.where(np.arange(n) < n // 2, -1.0, 1.0))  # two n/2-fold levels
    A = with_spectrum(rng, rows)
    check(ctxs[form], A, form, f"degenerate / near-degenerate n={n}")
    # zero, diagonal, rank one, tiny and huge scales
    Z = np.zeros((1, n, n), dtype=np.complex128)
    D = np.diag(rng.normal(size=n)).astype(np.complex128)[None]
    u = rng.normal(size=n) + 1j * rng.normal(size=n)
    R1 = np.outer(u, np.conj(u))[None]
    H = rand_herm(rng, 2, n)
    check(ctxs[form], np.concatenate([Z, D, R1, 1e-30 * H[:1], 1e30 * H[1:]]), form, f"special n={n}")


def test_device_pointers_and_errors(ctxs):
    torch = pytest.importorskip("torch")
    wl = synth.make_workload("si_tiny", nk=4, nq=2)
    ctx = binding.Context.from_workload(wl, device_ptrs=True)
    rng = np.random.default_rng(7)
    A = rand_herm(rng, 33, 10)
    dA = torch.from_numpy(A).cuda()
    dw = torch.empty(33, 10, dtype=torch.float64, device="cuda")
    dV = torch.empty(33, 10, 10, dtype=torch.complex128, device="cuda")
    ctx.eph_eigh(10, 33, dA, dw, dV)
    torch.cuda.synchronize()
    w_ref, _ = oracle.electron_eigen(A)
    assert np.abs(dw.cpu().numpy() - w_ref).max() <= 1e-13 * np.abs(w_ref).max()
    with pytest.raises(binding.EphError) as ei:
        ctx.eph_eigh(257, 1, dA, dw, dV)
    assert ei.value.code == binding.EPH_EINVAL
    with pytest.raises(binding.EphError):
        ctx.eph_eigh(10, 0, dA, dw, dV)
    # V carries intermediate results: an in-place call is rejected, not silently wrong
    with pytest.raises(binding.EphError) as ei:
        ctx.eph_eigh(10, 33, dA, dw, dA)
    assert ei.value.code == binding.EPH_EINVAL


@pytest.mark.parametrize("n,plain,kernels", [(8, False, 2), (11, False, 2), (14, False, 1), (8, True, 1)])
def test_launch_count_is_the_kernels_launched(n, plain, kernels):
    # the context counts every kernel each of its calls enqueues (the bench's gpu_launches):
    # n <= 12 runs the FP32 sweeps and the refinement as two kernels, n = 13..16 and the plain
    # FP64 option one
    wl = synth.make_workload("si_tiny", nk=4, nq=2)
    ctx = binding.Context.from_workload(wl, eig_plain_fp64=plain)
    A = rand_herm(np.random.default_rng(n), 40, n)
    before = ctx.launches()
    ctx.eigh(A)
    assert ctx.launches() - before == kernels
