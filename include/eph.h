/*
 * libeph: Wannier interpolation of electron-phonon matrix elements on one GB300.
 *
 * The library computes, for fine k and q points, the quantities of the paper's
 * nested-loop algorithm (arxiv 2603.10295, section "Analysis of computational
 * complexity", Eqs. 9-10, which refactor the interpolation formula Eq. 7):
 *
 *   eps_nk, U_k       eigenpairs of H(k)   = sum_Re w_e e^{i k.Re} H(Re)
 *   omega_qnu, e_qnu  eigenpairs of D(q)   = sum_Rp w_p e^{i q.Rp} Phi(Rp)/sqrt(M M')
 *   g(Re,q)           = sum_Rp e^{i q.Rp} g(Re,Rp)                          (Eq. 9)
 *   g_mnnu(k,q)       = sum U_{mm',k+q} U*_{nn',k} u_{ka,nu}(q) e^{i k.Re} g(Re,q)   (Eq. 10)
 *
 * Conventions:
 *   - e^{i k.R} = exp(2 pi i sum_j k_j n_j), k in crystal (reciprocal-basis)
 *     coordinates, R = (n1,n2,n3) integer lattice coordinates; the argument is
 *     formed in FP64 and reduced exactly (t - rint(t)) before sincospi.
 *   - U_{nn'k} = conj(V_k[n'][n]) where V_k holds the eigenvectors of H(k) as
 *     columns in ascending eigenvalue order, so g_nu(k,q) = V_{k+q}^H G V_k.
 *   - u_{ka,nu}(q) = e_{ka,nu}(q)/sqrt(M_kappa) (M in amu), index ka = 3*kappa+alpha.
 *   - omega = sign(lambda) sqrt(|lambda|) * hbar sqrt(eV/(A^2 amu)) in eV.
 *   - complex numbers are (re, im) pairs of doubles (complex128) or floats (complex64).
 *
 * Errors: every entry point returns EPH_OK (0) or a negative code; a per-context
 * message is available from eph_last_error.  Nothing exits or throws across
 * the ABI.  A context is not thread-safe: calls on one context must not run
 * concurrently; they are ordered on the context's CUDA stream.
 */
#ifndef EPH_H
#define EPH_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct eph_ctx eph_ctx;

enum eph_status {
  EPH_OK = 0,
  EPH_EINVAL = -1,    /* bad argument: NULL pointer, non-positive or unsupported size */
  EPH_ENOMEM = -2,    /* device allocation failed */
  EPH_ECUDA = -3,     /* a CUDA runtime call or kernel launch failed */
  EPH_ENOTCONV = -4,  /* a batched Jacobi eigensolve hit its sweep cap */
  EPH_ESTATE = -5,    /* call out of order (e.g. eph_interp_q before eph_set_k) */
  EPH_ENOTSUP = -6    /* size or form the library does not support */
};

enum eph_form {
  EPH_FORM_FP64 = 0,  /* every result to FP64 accuracy: FP64 DFMA, except the band rotation
                         (nb <= 16, nm*nb <= 128) and, on k lists, the Re->k contraction with
                         H(k+q) (2 ne <= 512, nb, nm <= 16), which run on the tensor cores from
                         six- or seven-digit fixed-point BF16 operands with exact level sums and
                         integer-assembled doubles (~1e-13 of each pair's or column's largest
                         term; options band_alu and gemm_alu select DFMA) */
  EPH_FORM_MIXED = 1  /* split precision on the large contractions, g as complex64: on k lists the
                         Re->k contraction of g and H(k+q) are tcgen05 tensor-core products of
                         fixed-point BF16 digits with FP32 accumulation; the Rp->q contraction
                         (Eq. 9) is one too while its digit planes stay below ~4 GB (Si- and
                         MoS2-shaped inputs; FP64 otherwise); the band rotation runs on the tensor
                         cores (fused two-product kernel for nb <= 16, nm*nb <= 128; batched
                         products beyond; option band_alu selects double-float FP32 for the former);
                         the eigensolves stop at eigenvalues within ~1e-12 ||A|| and eigenvectors
                         within ~1e-8.  Phases (exact FP64 reduction), D(q) and its eigensolve and,
                         on uniform grids, the Re->k transforms stay FP64 */
};

typedef struct eph_options {
  int form;          /* enum eph_form */
  int device_ptrs;   /* 0: k/q lists and outputs are host pointers (the call copies and
                        synchronises); 1: they are device pointers (CUDA-visible memory) */
  int q_batch;       /* q points per internal batch, 0 = automatic */
  int k_tile;        /* k points per internal tile, 0 = automatic (bounded by workspace_mb) */
  int max_sweeps;    /* Jacobi sweep cap, 0 = default (20) */
  int workspace_mb;  /* soft cap on the per-call workspace in MiB, 0 = default (4096) */
  int mixed_scheme;  /* mixed form only: 0 = fixed-point BF16 digits (3 for the phases, 4 for g)
                        with exact FP32 tensor-core accumulation (default; needs 2*ne <= 1024),
                        1 = two-term split TF32 (3 products) */
  int eig_plain_fp64; /* 0 (default): FP32 Jacobi sweeps, then refinement to full FP64 accuracy
                         (n <= 12: Ogita-Aishima steps, the first in double-float on the FP32 pipe,
                         the last in FP64; plain FP64 sweeps for n = 13..16; Newton-Schulz,
                         A' = V^H A V and FP64 polish sweeps for n > 16);
                         1: plain FP64 Jacobi sweeps only */
  int async;          /* 1: eph_interp_q only enqueues work (no host synchronisation, no event
                         timing); its status is read by eph_sync.  With device pointers a sequence
                         of calls can be captured into one CUDA graph.  With host pointers (FP64
                         form, uniform-grid path or nb, nm > 16) the outputs are copied to the host
                         asynchronously, g on a second stream: the host buffers must stay valid,
                         and should be pinned, until eph_sync returns */
  int band_alu;       /* nb <= 16 and nm*nb <= 128: 0 (default) = band rotation on the tensor cores,
                         fixed-point BF16 digit products with exact level sums (mixed form: four
                         digits per operand, ~2^-31 of each pair's largest element; FP64 form: six
                         digits, levels <= 6, integer assembly of the doubles, ~1e-14); 1 = on the
                         CUDA cores (double-float FP32 in the mixed form, FP64 DFMA in the FP64
                         form).  The same switch applies to the FP64 band products of
                         eph_interp_backward, eph_interp_vjp, eph_bloch_to_wannier and
                         eph_linewidths (six-digit tensor-core products, or FP64 DFMA) */
  int gemm_alu;       /* the FP64-accuracy GEMMs: the Re->k contraction of Eq. 10 on a k list (FP64
                         form and every FP64 chain; 2 ne <= 512, nb, nm <= 16), Eq. 9 (2 Np <= 512,
                         digit planes of g(Re,Rp) within 1/16 of the device), the adjoint's gradient
                         GEMM, and the mixed form's mode rotation for nm > 16: 0 (default) = on the
                         tensor cores, seven balanced base-128 digits per operand (power-of-two
                         scale per row and per column), exact level sums, doubles assembled from
                         64-bit integers (~1e-14 of each column's largest term); 1 = FP64 DFMA
                         (double-float for the mixed form's mode rotation) */
} eph_options;

/* Fills *opt with the defaults (FP64 form, host pointers, automatic batching). */
void eph_default_options(eph_options* opt);

/*
 * Creates a context on the current CUDA device and uploads the Wannier-space
 * data (paper Eq. 3 and the electron/phonon Wannier Hamiltonians).
 *
 *   nb, na           Wannier functions and atoms per cell; nm = 3*na modes.
 *   ne, np           number of electron (Re) and phonon (Rp) lattice vectors.
 *   H_Re    [ne][nb][nb] complex128, eV      H(Re) = <w_m0|H|w_nRe>
 *   Phi_Rp  [np][nm][nm] double, eV/A^2     force constants Phi_{ka,k'b}(Rp)
 *   g_ReRp  [np][nm][ne][nb][nb] complex128, eV   g_{m'n'ka}(Re,Rp) (Eq. 3),
 *                                           16*nb*nb*nm*ne*np bytes (Table 3 caption)
 *   Re [ne][3], Rp [np][3]  integer lattice coordinates
 *   we [ne], wp [np]        per-vector weights (Wigner-Seitz degeneracies); NULL = all 1
 *   masses [na]             amu
 *   opt                     NULL = defaults
 *   cuda_stream             cudaStream_t to order all work on; NULL = a stream the
 *                           context creates and owns
 * All inputs are HOST pointers; they are copied and may be freed on return.
 * Supported sizes: 1 <= nb, nm <= 16 (warp-resident Jacobi and rotations) and up to
 * 256 (one CTA per eigensolve, GEMM rotations; forward only), in both forms (beyond 16
 * the FP64 form rotates with batched FP64 GEMMs; the mixed form runs the Re->k contraction,
 * H(k+q) and the band rotation on the tensor cores, the mode rotation and the eigensolves'
 * products in double-float); larger sizes return EPH_ENOTSUP.  The mixed form's digit
 * scheme (mixed_scheme 0) needs 2*ne <= 1024 (EPH_ENOTSUP otherwise).
 * On success *out owns device memory until eph_destroy.
 */
int eph_create(eph_ctx** out, int nb, int na, int ne, int np,
               const double* H_Re, const double* Phi_Rp, const double* g_ReRp,
               const int* Re, const double* we, const int* Rp, const double* wp,
               const double* masses, const eph_options* opt, void* cuda_stream);

/*
 * Sets the fine k list: phases e^{i k.Re}, H(k) and its batched FP64
 * eigensolve stay resident on the device for later eph_interp_q calls.
 *   kpts  [nk][3] crystal coordinates        (host or device, see device_ptrs)
 *   eps_k [nk][nb] eV ascending, may be NULL (host or device)
 */
int eph_set_k(eph_ctx* ctx, int nk, const double* kpts, double* eps_k);

/*
 * Sets the fine k list to the uniform grid k = (j1/n1, j2/n2, j3/n3) + shift, k index
 * (j1 n2 + j2) n3 + j3 (j3 fastest), and computes what eph_set_k computes for it.
 * On such a grid the phase of Eq. 10 (and of the H(k+q) sum of Eq. 4) factorises per
 * axis, e^{2 pi i k.Re} = prod_a e^{2 pi i k_a n_a}, so later eph_interp_q,
 * eph_linewidths calls evaluate the Re->k contraction as three one-axis transforms over
 * the bounding box of the Re list (B_a terms per output instead of ne): the same sum,
 * term for term, to rounding.  Used when nb, nm <= 16, the Re vectors are distinct and
 * their box has extents <= 32 and volume <= 8 ne; otherwise the general path runs on the
 * generated k list.  In the mixed form the transforms are FP64 as well; the band rotation
 * runs on the tensor cores from these FP64 sums (rounded to FP32) and the eigensolves stop at
 * the mixed form's accuracy (g complex64).
 *   shift [3] HOST pointer (NULL = 0); eps_k [nk][nb] as in eph_set_k (may be NULL).
 * EPH_EINVAL for n_a < 1 or nk > 2^31 - 1.
 */
int eph_set_k_grid(eph_ctx* ctx, int n1, int n2, int n3, const double* shift, double* eps_k);

/*
 * Interpolates for nq q points against the resident k list (paper Eqs. 9-10
 * with the D(q) and H(k+q) eigensolves).
 *   qpts   [nq][3] crystal coordinates
 *   eps_kq [nq][nk][nb] eV (eigenvalues of H(k+q)), may be NULL
 *   omega  [nq][nm] eV, may be NULL
 *   g      [nq][nk][nm][nb][nb]: complex128 in the FP64 form, complex64 in the
 *          mixed form; may be NULL (then only eps_kq/omega are produced)
 * Returns EPH_ESTATE if eph_set_k has not been called.
 */
int eph_interp_q(eph_ctx* ctx, int nq, const double* qpts, double* eps_kq, double* omega, void* g);

/*
 * Rp-partitioned g(Re,Rp) (the paper's "Workload distribution": pools split the Rp vectors of
 * g(Re,Rp) and sum the partial Eq. 9 results over the pool before the k stage).  For a
 * g(Re,Rp) larger than one GPU's memory (Table 3's widest ribbons: 353-458 GiB), each GPU holds
 * the slice Rp[rp_begin .. rp_begin + rp_count - 1]:
 *
 *   eph_create_rp_slice  as eph_create, but g_ReRp_slice is [rp_count][nm][ne][nb][nb]
 *                        complex128, the rows of g(Re,Rp) for that Rp range.  Phi_Rp, Rp and wp
 *                        still cover all np vectors (D(q) needs every force constant).
 *                        EPH_EINVAL unless 0 <= rp_begin, 1 <= rp_count, rp_begin + rp_count <= np.
 *   eph_g1_partial       G1 [nq][nm][ne][nb][nb] complex128 = sum over the slice's Rp of
 *                        w_p e^{i q.Rp} g(Re,Rp) (Eq. 9 restricted to the slice); the sum of
 *                        the partials of all slices (an allreduce across the GPUs) is Eq. 9.
 *   eph_interp_q_g1      eph_interp_q with G1 [nq][nm][ne][nb][nb] complex128 supplied by the
 *                        caller (the summed partials) in place of Eq. 9: outputs as eph_interp_q.
 *                        Works on any context (also a whole one).
 * qpts, G1 and the outputs are host or device pointers per device_ptrs.  On an Rp-slice context
 * (rp_count < np) eph_interp_q, eph_interp_q_window, eph_interp_backward and eph_linewidths,
 * which would need the whole Eq. 9, return EPH_ESTATE; eph_interp_vjp and eph_bloch_to_wannier
 * do not read g(Re,Rp) and return the whole [np] result.
 */
int eph_create_rp_slice(eph_ctx** out, int nb, int na, int ne, int np, const double* H_Re, const double* Phi_Rp,
                        const double* g_ReRp_slice, const int* Re, const double* we, const int* Rp, const double* wp,
                        const double* masses, int rp_begin, int rp_count, const eph_options* opt, void* cuda_stream);
int eph_g1_partial(eph_ctx* ctx, int nq, const double* qpts, double* G1);
int eph_interp_q_g1(eph_ctx* ctx, int nq, const double* qpts, const double* G1, double* eps_kq, double* omega,
                    void* g);

/*
 * Replaces the resident g(Re,Rp) (or the context's Rp slice of it) by g_ReRp, same layout as at
 * creation ([nrp][nm][ne][nb][nb] complex128), host or device pointer per device_ptrs; the
 * Hamiltonians, force constants and the resident k list are kept.  A device-to-device copy in
 * device mode: this is how a training loop feeds an updated g(Re,Rp) tensor back to the same
 * context without a host round trip.
 */
int eph_set_gw(eph_ctx* ctx, const double* g_ReRp);

/*
 * eph_interp_q for several contexts (materials of different nb, nm, each with its own q batch of
 * any size) in one call whose band rotations run as persistent kernels over a mixed work list:
 * the calls proceed in rounds, each context contributing its next (q batch, k tile) unit (phases,
 * D(q), Eq. 9 and the mode rotation at the start of a q batch; the Re->k contraction and the
 * H(k+q) eigensolves per tile), and one launch per round rotates the pairs of every context's
 * unit, its CTAs walking the concatenated pair list (k_band_rotate_multi, the FP64 DFMA rotation).
 * Results are bit for bit those of separate eph_interp_q calls on contexts created with
 * band_alu = 1; the default separate calls rotate on the tensor cores and agree to ~5e-14 of each
 * pair's largest |g|.
 *   ctxs[nctx] distinct contexts, 1 <= nctx <= 32, each with a resident k list, FP64 form,
 *   nb, nm <= 16, device pointers, whole g(Re,Rp) (else EPH_ENOTSUP); nq[i], qpts[i], eps_kq[i],
 *   omega[i], g[i] as eph_interp_q's arguments for context i (eps_kq, omega, g and their
 *   entries may be NULL).
 * All the work runs on ctxs[0]'s stream (it first waits for the work queued on the other
 * contexts' streams, which wait for the call at its end); with every context on one stream the
 * call can be captured into a CUDA graph (async mode).  Errors are reported on ctxs[0].
 */
int eph_interp_q_multi(int nctx, eph_ctx* const* ctxs, const int* nq, const double* const* qpts,
                       double* const* eps_kq, double* const* omega, void* const* g);

/* eph_set_k followed by eph_interp_q. */
int eph_interp(eph_ctx* ctx, int nk, const double* kpts, int nq, const double* qpts,
               double* eps_k, double* eps_kq, double* omega, void* g);

/*
 * Scalar L = sum_{q,k,nu,m,n} w_nk |g_mnnu(k,q)|^2 / omega_qnu over modes with
 * omega_qnu > omega_min, and its gradient with respect to g(Re,Rp) with the
 * eigenvectors U and e held fixed (hand-written adjoint of Eqs. 9-10; the
 * Re->k stage is recomputed, never stored).
 *   w_nk         [nk][nb] weights (host or device per device_ptrs)
 *   L_out        one double (host or device)
 *   grad_g_ReRp  [np][nm][ne][nb][nb] complex128, dL/dRe(g) + i dL/dIm(g)
 *                (the PyTorch convention for a real scalar of complex inputs)
 * Uses the k list given here (it replaces the resident one).  kpts = NULL: the resident k
 * list (nk must equal its size); after eph_set_k_grid both Re->k sums -- the recomputed
 * forward one and its adjoint -- then run sum-factorised, as three one-axis transforms
 * (the adjoint applies the conjugate axis phases in reverse order and gathers the Re rows).
 * Every supported shape and both forms: the chain is FP64 (a mixed-form context recomputes
 * the forward with the FP64 Eq. 9, its electron eigensolves polished to 1e-12).  The band
 * rotation and its adjoint run on the tensor cores at FP64 accuracy (six-digit operands,
 * ~5e-14 of each pair's largest element) for nb <= 16, nm nb <= 128 unless band_alu is set,
 * as FP64 GEMMs batched over (k, nu) for larger shapes.  An Rp-slice context returns
 * EPH_ESTATE.
 */
int eph_interp_backward(eph_ctx* ctx, int nk, const double* kpts, int nq, const double* qpts,
                        const double* w_nk, double omega_min, double* L_out, double* grad_g_ReRp);

/*
 * Vector-Jacobian product of the interpolation (the adjoint chain of Eqs. 9-10 and the
 * band rotation of Eq. 7, applied to an arbitrary upstream gradient): with U_k, U_{k+q}
 * and e_q held fixed, g(k,q) is linear in g(Re,Rp), and
 *   grad_g_ReRp = A^H grad_g,   A: g(Re,Rp) -> g(k,q) of eph_interp_q,
 * i.e. for a real scalar L(g) and grad_g = dL/dRe(g) + i dL/dIm(g) (PyTorch convention)
 * it returns dL/dRe(gW) + i dL/dIm(gW).  The gauges are recomputed bit for bit as
 * eph_set_k / eph_interp_q produce them for the same context, so grad_g must refer to g
 * as this context returned it.
 *   kpts [nk][3], qpts [nq][3]; grad_g [nq][nk][nm][nb][nb] complex128; grad_g_ReRp
 *   [np][nm][ne][nb][nb] complex128 (overwritten).  Host or device pointers per
 *   device_ptrs.  Replaces the context's k list (as eph_set_k); kpts = NULL keeps the
 *   resident one (sum-factorised on a uniform grid, as in eph_interp_backward).
 * Every supported shape and both forms (an FP64 chain, as eph_interp_backward; in a mixed-form
 * context the gauges are that context's, its electron eigensolves polished to 1e-12).
 */
int eph_interp_vjp(eph_ctx* ctx, int nk, const double* kpts, int nq, const double* qpts, const void* grad_g,
                   double* grad_g_ReRp);

/*
 * Bloch -> Wannier transform of Eq. 6 (the coarse-grid construction that precedes the
 * interpolation): for g_mnnu(k',q') given on nk coarse k' and nq coarse q' points in the
 * gauges this context's H(Re), Phi(Rp) define (U_k', U_k'+q', u_q' as eph_interp_q uses them),
 *   g(Re,Rp) = 1/(ne np) sum_{k',q'} e^{-i(k'.Re + q'.Rp)} sum_nu u^{-1}_{nu,ka}(q')
 *              [U_{k'+q'} g_nu(k',q') U_{k'}^H]  (U in the eigenvector-column convention),
 * the exact inverse of the interpolation when k' and q' run over the Born-von Karman grid
 * whose supercell vectors are Re = Rp (unit weights; weights are not used here).
 *   kpts [nk][3], qpts [nq][3]; g [nq][nk][nm][nb][nb] complex128; g_ReRp [np][nm][ne][nb][nb]
 *   complex128 (overwritten).  Host or device pointers per device_ptrs.  Replaces the
 *   context's k list (as eph_set_k); kpts = NULL keeps the resident one (e.g. the coarse grid
 *   set by eph_set_k_grid, whose sums over k' then run sum-factorised).  The context's own
 *   g(Re,Rp) is not used.
 * Every supported shape and both forms (an FP64 chain, as eph_interp_vjp).
 */
int eph_bloch_to_wannier(eph_ctx* ctx, int nk, const double* kpts, int nq, const double* qpts, const void* g,
                         double* g_ReRp);

/*
 * Energy-window prescreening of the fine k list (the paper's transport workflow drops the k
 * points whose states all lie outside a window around the band edge before forming g):
 * computes eps_nk for all nk points of kpts, keeps the points with some band in
 * [e_lo, e_hi], and makes the kept points, in their input order, the resident k list (as
 * eph_set_k with that list would).
 *   kpts [nk][3]; eps_k [nk_kept][nb] of the kept points (may be NULL); kidx [nk] receives the
 *   kept indices into kpts (first *nk_kept entries); host or device pointers per
 *   device_ptrs; *nk_kept on the host.  With nothing in the window *nk_kept = 0 and no k list
 *   is resident.  Reads the kept count on the host: not available in async mode.
 */
int eph_set_k_window(eph_ctx* ctx, int nk, const double* kpts, double e_lo, double e_hi, double* eps_k,
                     int* kidx, int* nk_kept);

/*
 * Irreducible k list of a uniform grid under time reversal (the paper's transport workflow
 * interpolates on the irreducible wedge of the fine k grid with weights, then prescreens it by
 * the energy window): for Hamiltonians whose H(Re) are real (H(-Re) = H(Re)^T), H(-k) =
 * conj H(k), so eps(-k) = eps(k) and a k-sum over the grid equals the weighted sum over one
 * point of each pair {k, -k}.  Grid point i = (j1 n2 + j2) n3 + j3 at k = j/n + shift; its
 * partner -k is grid point (-j_a - 2 shift_a n_a) mod n_a; i is kept if i <= its partner,
 * with weight 2 (1 if it is its own partner).  The kept points, ascending, become the resident
 * k list (a plain list: later Re->k sums use the general path).
 *   shift [3] HOST pointer (NULL = 0); 2 shift_a n_a must be an integer on every axis (else
 *   EPH_EINVAL).  eps_k [nk_kept][nb] (may be NULL), kidx [n1 n2 n3] receives the kept grid
 *   indices (first *nk_kept entries), wk [n1 n2 n3] their weights (sum = n1 n2 n3); host or
 *   device pointers per device_ptrs; *nk_kept on the host.  Not available in async mode.
 * The reduction is pure index arithmetic (bit-exact); whether H(Re) has the symmetry is the
 * caller's to know (the library does not check it).
 */
int eph_set_k_grid_ibz(eph_ctx* ctx, int n1, int n2, int n3, const double* shift, double* eps_k, int* kidx,
                       double* wk, int* nk_kept);

/*
 * eph_interp_q with pair screening: pairs (q,k) with no eps_{m,k+q} in [e_lo, e_hi] get g = 0
 * without the band rotation (the only step after eps_{k+q} is known); keep [nq][nk] (int, may
 * be NULL) receives 1 for the pairs computed and 0 for the screened ones.  eps_kq and omega are
 * complete.  Both forms (g complex64 in the mixed form) and every supported shape: for nb,
 * nm <= 16 the screened pairs skip the band rotation (its kernels write their g as 0); beyond,
 * every pair is rotated and the screened ones are zeroed afterwards (no work saved).
 */
int eph_interp_q_window(eph_ctx* ctx, int nq, const double* qpts, double e_lo, double e_hi, double* eps_kq,
                        double* omega, void* g, int* keep);

/*
 * Electron linewidths from the interpolated couplings without writing g (a fused
 * downstream consumer; the paper's mobility and self-energy workloads consume g this
 * way): for the resident k list and nq q points,
 *   gamma[k][n] = pi sum_q w_q sum_{m, nu: omega_qnu > omega_min} |g_mnnu(k,q)|^2 / (2 omega_qnu)
 *     x [ (n_B(omega) + f(e_{m,k+q})) delta(e_nk - e_{m,k+q} + omega)
 *       + (n_B(omega) + 1 - f(e_{m,k+q})) delta(e_nk - e_{m,k+q} - omega) ]
 * with n_B = 1/(exp(omega/kT) - 1), f = 1/(exp((e - mu)/kT) + 1) and a Gaussian delta of
 * width sigma (all in eV); g as eph_interp_q defines it.  Units: |g|^2 / eV^2.
 *   qpts [nq][3], wq [nq] q weights (NULL = all 1), gamma [nk][nb] (overwritten with the
 *   sum over these q points); host or device pointers per device_ptrs.
 * Every supported shape and both forms, in FP64 (a mixed-form context runs the FP64 chain with
 * its electron eigensolves polished to 1e-12).  g is formed over the context's k-tile
 * workspace and reduced there: by the FP64-accuracy tensor-core rotation for nb <= 16,
 * nm nb <= 128 (the fused CUDA-core kernel with band_alu), by FP64 GEMMs for larger shapes.
 * An Rp-slice context returns EPH_ESTATE.
 */
int eph_linewidths(eph_ctx* ctx, int nq, const double* qpts, const double* wq, double kT, double mu,
                   double sigma, double omega_min, double* gamma);

/* Releases every device resource of the context (NULL is a no-op). */
void eph_destroy(eph_ctx* ctx);

/* Static description of a status code. */
const char* eph_strerror(int code);

/* Message of the last failing call on this context ("" if none). */
const char* eph_last_error(const eph_ctx* ctx);

/* Number of kernels this context has launched since creation (instrumentation). */
long long eph_kernel_launches(const eph_ctx* ctx);

/* Stages of the pipeline, for per-stage kernel timing. */
enum eph_stage {
  EPH_STAGE_PHASE = 0, /* phase factors e^{i k.R} (exact FP64 reduction + sincospi)             */
  EPH_STAGE_FT_Q = 1,  /* Rp->q contraction of g (Eq. 9) and D(q)                              */
  EPH_STAGE_EIG = 2,   /* batched Hermitian Jacobi eigensolves of H(k), H(k+q)                   */
  EPH_STAGE_MODE = 3,  /* D(q) eigensolve, mode rotation by u(q), per-q operand assembly
                          (on a product k grid also the axis-3 and axis-2 transforms)        */
  EPH_STAGE_FT_K = 4,  /* Re->k contraction (Eq. 10 Fourier sum) fused with H(k+q); on a
                          product k grid its per-k part, the axis-1 transform              */
  EPH_STAGE_BAND = 5,  /* band rotation V_{k+q}^H G V_k (in eph_interp_backward: its adjoint
                          V_{k+q} (2 c g) V_k^H with the loss terms)                       */
  EPH_STAGE_ADJ = 6,   /* the other adjoint (backward) kernels                                  */
  EPH_STAGE_TC = 7,    /* mixed form: tensor-core (tcgen05) Re->k contraction                   */
  EPH_NSTAGES = 8
};

/*
 * enable != 0: every kernel the context launches is bracketed by CUDA events
 * on the context's stream and its duration is added to its stage when the
 * call completes.  eph_profile_read returns the accumulated milliseconds and
 * launch count of one stage; eph_profile_reset clears them.
 */
int eph_profile(eph_ctx* ctx, int enable);
int eph_profile_read(const eph_ctx* ctx, int stage, double* ms, long long* launches);
int eph_profile_reset(eph_ctx* ctx);

/*
 * Batching support (several materials / uneven q batches in one captured CUDA graph):
 *   eph_reserve   sizes every workspace buffer for calls of up to nq q points with the
 *                 resident k list, so that later eph_interp_q calls allocate nothing
 *                 (a requirement for stream capture).
 *   eph_sync      synchronises the context's streams (its own and the one that copies g to
 *                 host buffers), reads and clears the device status flags of the work
 *                 enqueued since the last check (async mode).
 *   eph_autotune  picks q_batch and k_tile for nq q points by timing candidate
 *                 decompositions (q_batch 1..16, k tiles of nk, nk/2, nk/4) with CUDA
 *                 events on the context's stream, then, at that decomposition, the kernel
 *                 variants band_alu and gemm_alu (each must be 3 % faster than the
 *                 tensor-core default to replace it; both meet the form's accuracy);
 *                 the choice is applied to the context's options and cached per problem
 *                 shape and device (name, SM count) for the process, and in the tuning
 *                 file if one is set.  Needs device pointers and synchronous mode;
 *                 allocates its probe outputs.
 *   eph_tune_file sets the process's tuning file (NULL: none) and clears the process
 *                 cache; reads the file if it exists (entries of other devices are kept
 *                 but never match).  Returns the number of entries read, or EPH_EINVAL for
 *                 a malformed line (the cache stays empty).  Timed entries are appended.
 *                 Line format: "eph-tune 1 <device, spaces as _> <SMs> <form> <scheme>
 *                 <grid> <nb> <nm> <ne> <np> <nk> <nq> : <q_batch> <k_tile> <band_alu>
 *                 <gemm_alu>"; lines starting with # are comments.  No CUDA call.
 *   eph_tuning    the context's current choice and where it came from.
 */
typedef struct {
  int q_batch, k_tile, band_alu, gemm_alu;
  int source; /* 0: not tuned, 1: timed by eph_autotune, 2: this process's cache, 3: the tuning file */
} eph_tuning_info;
int eph_reserve(eph_ctx* ctx, int nq);
int eph_sync(eph_ctx* ctx);
int eph_autotune(eph_ctx* ctx, int nq, const double* qpts, int* q_batch_out, int* k_tile_out);
int eph_tune_file(const char* path);
int eph_tuning(const eph_ctx* ctx, eph_tuning_info* out);

/*
 * The batched Hermitian eigensolver of the interpolation, on caller matrices: the
 * diagonalisations of Eq. 4 (H(k), H(k+q) -> eigenvalues eps and the gauge columns U) and
 * Eq. 5 (D(q) -> omega^2 and the mode eigenvectors) as one call.
 *   A     [batch][n][n] complex128 (re, im), row-major; only the Hermitian part is used
 *         (the imaginary parts of the diagonal are ignored).
 *   w     [batch][n] eigenvalues, ascending (ties in input order).
 *   V     [batch][n][n] complex128, column j the unit eigenvector of w[j] (V^H A V = diag w);
 *         it holds intermediate results during the call, so it must not overlap A.
 * Host or device pointers per the context's device_ptrs option; the call runs on the
 * context's stream and is synchronous unless the context is in async mode.
 * 1 <= n <= 256, batch >= 1.  Precision follows the context's form: FP64 eigenvalues and
 * eigenvectors (residual ~1e-15 ||A||) for EPH_FORM_FP64; for EPH_FORM_MIXED eigenvalues
 * within ~1e-12 ||A|| and eigenvectors within ~1e-8.  eig_plain_fp64 selects the plain FP64
 * Jacobi sweeps.  Errors: EPH_EINVAL (sizes, NULL pointers, A and V overlapping), EPH_ENOTCONV (a matrix reached
 * max_sweeps; results still written), EPH_ENOMEM, EPH_ECUDA.
 */
int eph_eigh(eph_ctx* ctx, int n, int batch, const void* A, double* w, void* V);

/*
 * Band energies and eigenvectors of H(k) = sum_Re w_e e^{i k.Re} H(Re) for a
 * k list, computed without any device allocation by the library.  The paper
 * has no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- processes whose device memory is owned by another allocator
 * (a framework's caching allocator that reserved the HBM up front, an
 * embedding application with a fixed budget) and latency-sensitive callers
 * that must not trigger the device-wide synchronisation cudaMalloc/cudaFree
 * can cause.  It runs the same kernels as eph_set_k, with their scratch
 * (the phases and the H(k) matrices) in one fixed device array of
 * EPH_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until
 * the process exits.
 *
 *   kpts [nk][3] f64, Re [ne][3] int32, we [ne] f64 (NULL = all 1),
 *   H_Re [ne][nb][nb] complex128: DEVICE pointers, read only.
 *   eps  [nk][nb] f64 ascending, U [nk][nb][nb] complex128 (eigenvectors as
 *   columns): DEVICE pointers, written.
 *   max_sweeps: Jacobi sweep cap, <= 0 = 20.  cuda_stream: stream to run on (NULL = legacy default).
 * Limits: 1 <= nb <= 16 and scratch = round_up(16*nk*ne, 256) + 16*nk*nb*nb
 * bytes <= EPH_NOALLOC_SCRATCH_BYTES, else EPH_EINVAL before any GPU work.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, once per device, with that device current; again
 * if the current CUDA context changed, e.g. after cudaDeviceReset); make
 * that first call before any stream capture.  The call synchronises the
 * stream to report the eigensolver status (EPH_ENOTCONV at the sweep cap):
 * it blocks the calling host thread until all work queued on that stream,
 * including work queued before the call, has finished.
 * All calls share the one array and it keeps the last call's contents: calls
 * that overlap on the GPU (other streams or host threads on the same device)
 * race and must be serialised by the caller.
 */
#define EPH_NOALLOC_SCRATCH_BYTES (32u << 20)
int eph_bands_noalloc(int nk, const double* kpts, int nb, int ne, const int* Re, const double* we,
                      const double* H_Re, double* eps, double* U, int max_sweeps, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* EPH_H */
