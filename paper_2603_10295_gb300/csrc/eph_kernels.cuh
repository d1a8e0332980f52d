// Internal launch interface of the libeph CUDA kernels (sm_103a).
// Every launcher enqueues on `st` and returns cudaGetLastError() of the launch.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace eph {

// ---- launch accounting --------------------------------------------------------
// Every kernel launch site counts itself (kernels enqueued by this host thread); a context adds
// the difference over each of its calls to its launch count.
extern thread_local long long t_kernel_launches;
inline void note_launch() { ++t_kernel_launches; }

// ---- complex helpers (double2 / float2 = re, im) ---------------------------
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__host__ __device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

// ---- phases (paper Eq. 7 factors e^{i k.Re}, e^{i q.Rp}) --------------------
// P[i*ldp + r] = w[r] * exp(2 pi i pts_i . R_r); w may be null (weight 1).
cudaError_t launch_phase(const double* pts, int n, const int* R, const double* w, int nR,
                         double2* P, long ldp, cudaStream_t st);
// B[q][e][j] = Q[q][e] * H[e][j] for j < cols; output row stride ldb, batch stride sB.
cudaError_t launch_scale_rows(const double2* Q, int nq, const double2* H, int ne, int cols,
                              double2* B, long ldb, long sB, cudaStream_t st);

// ---- FP64 complex GEMM: C[b] = A[b] * B[b], row-major -----------------------
// A: M x K (lda, batch stride sA, may be 0), B: K x N (ldb, sB), C: M x N (ldc, sC).
cudaError_t launch_zgemm(int M, int N, int K, const double2* A, long lda, long sA,
                         const double2* B, long ldb, long sB, double2* C, long ldc, long sC,
                         int batch, cudaStream_t st);
// Two-level batch: z = b1 * nbat2 + b2, operand offsets b1*s + b2*s2; adj: op(A) = A^H (A stored K x M).
cudaError_t launch_zgemm_b2(int M, int N, int K, const double2* A, long lda, long sA, long sA2, const double2* B,
                            long ldb, long sB, long sB2, double2* C, long ldc, long sC, long sC2, int nbat1,
                            int nbat2, int adj, cudaStream_t st);
// out[b][j][i] = in[b][i][j] for a batch of n x n complex matrices.
cudaError_t launch_transpose(const double2* in, int n, long batch, double2* out, cudaStream_t st);
// Same product on the FP32 pipe in double-float arithmetic (~1e-13 relative), FP64 in/out.
cudaError_t launch_zgemm_df(int M, int N, int K, const double2* A, long lda, long sA, const double2* B, long ldb,
                            long sB, double2* C, long ldc, long sC, int batch, cudaStream_t st);
// double-float C = op(A) B with a two-level batch (b1 < nbat1, b2 < nbat2; offsets b1 s*1 + b2 s*2),
// op(A) = A^H when adj; C complex64 when out32 (ldc, sC, sC2 in elements of C)
cudaError_t launch_zgemm_df_b2(int M, int N, int K, const double2* A, long lda, long sA, long sA2, const double2* B,
                               long ldb, long sB, long sB2, void* C, long ldc, long sC, long sC2, int nbat1, int nbat2,
                               int adj, int out32, cudaStream_t st);
// Adjoint form C[b] = A[b]^H * B[b] (A stored M_A x K_A = K x M), accumulate if acc.
cudaError_t launch_zgemm_ah(int M, int N, int K, const double2* A, long lda, long sA,
                            const double2* B, long ldb, long sB, double2* C, long ldc, long sC,
                            int batch, int acc, cudaStream_t st);
// Skinny rows: C[m][x] = sum_r P[m][r] * B[r][x], m < M <= 16 (P row stride ldp).
cudaError_t launch_skinny(int M, long N, int K, const double2* P, long ldp, const double2* B, long ldb,
                          double2* C, long ldc, cudaStream_t st);
// Skinny with real right operand (force constants): C[m][x] = sum_r P[m][r] * Breal[r][x] * s[x]
cudaError_t launch_skinny_real(int M, long N, int K, const double2* P, long ldp, const double* B,
                               long ldb, const double* colscale, double2* C, long ldc, cudaStream_t st);

// ---- batched Hermitian eigensolver (cyclic parallel Jacobi, FP64) -----------
// A[b] at A + b*sA (n x n, row stride lda); eigenvalues ascending to w + b*sw,
// eigenvectors as columns to V + b*sV (n x n, row stride n). n <= 16.
// status: device int, OR-ed with 1 if a matrix hit max_sweeps.
cudaError_t launch_jacobi(const double2* A, long sA, long lda, int n, long batch, double* w, long sw,
                          double2* V, long sV, int max_sweeps, int* status, cudaStream_t st);

// Same contract; FP32 preconditioning sweeps, two FP64 Newton-Schulz re-orthonormalisations,
// then FP64 sweeps to an off-diagonal norm <= polish_tol ||A||_F (n <= 12; larger n run the
// plain FP64 kernel).
cudaError_t launch_jacobi_mixed(const double2* A, long sA, long lda, int n, long batch, double* w, long sw,
                                double2* V, long sV, int max_sweeps, double polish_tol, int* status,
                                cudaStream_t st);

// 16 < n <= 256: one CTA per matrix, FP64 parallel Jacobi on a global working copy
// work [batch][n][n]; V must be packed (sV = n*n).
cudaError_t launch_jacobi_big(const double2* A, long sA, long lda, int n, long batch, double* w, long sw, double2* V,
                              long sV, double2* work, int max_sweeps, int* status, cudaStream_t st);
// Same contract, preconditioned: FP32 sweeps on a packed copy in shared memory, Newton-Schulz
// and A' = V^H A V as batched FP64 GEMMs, FP64 sweeps on A' to a first-order finish
// (polish_tol 1e-15: FP64 eigendecomposition; >= 1e-13: eigenvectors to ~1e-12).
// work: eigh_big_work_bytes(n, min(batch, 65535)) bytes.  eigh_big_supported(n): the packed
// FP32 copy fits in shared memory (n <= ~230 on GB300).
bool eigh_big_supported(int n);
size_t eigh_big_work_bytes(int n, long batch);
cudaError_t launch_eigh_big(const double2* A, long sA, long lda, int n, long batch, double* w, long sw, double2* V,
                            long sV, void* work, double polish_tol, int max_sweeps, int* status, cudaStream_t st);

// ---- phonon post-processing: omega = sign(l) sqrt|l| * unit; u = e / sqrt(M)
cudaError_t launch_phonon_post(const double* lam, const double2* e, int nq, int nm, const double* invsqrtm,
                               double unit, double* omega, double2* u, cudaStream_t st);

// ---- mode rotation: G2[q][e][nu][b] = sum_c u[q][c][nu] G1[q][c][e][b] -----------
// G2 written with row stride ldw (per e) and batch stride sW, starting at column 0.
cudaError_t launch_mode_rotate(const double2* G1, const double2* u, int nq, int nm, int ne, int nb2,
                               double2* W, long ldw, long sW, cudaStream_t st);

// ---- band rotation: g[q][k][nu] = Ukq[q][k]^H G3[q][k][nu] Uk[k] ---------------
// G3 rows: Y + (q*nk + k)*ldy (nm*nb*nb complex per row); Ukq [q][k][nb][nb];
// Uk [k][nb][nb]; output g + q*sgq + k*nm*nb*nb.
cudaError_t launch_band_rotate(const double2* Y, long ldy, const double2* Ukq, const double2* Uk, int nq,
                               int nk, int nm, int nb, double2* g, long sgq, cudaStream_t st,
                               const int* keep = nullptr);

// ---- Re->k contraction on a product k grid (sum factorisation, griddft.cu) ----------------
// kpts[(j1 n2 + j2) n3 + j3] = (j1/n1, j2/n2, j3/n3) + shift (shift: host array of 3)
// One segment of the persistent multi-material band rotation: pairs (q,k) of one (context,
// q batch, k tile), q-major with k fastest, first pair at global index pair0.
struct BandSeg {
  const double2* Y;    // G3 rows of the tile (pair p at Y + p * ldy)
  long ldy;
  const double2* Ukq;  // [pairs][nb][nb]
  const double2* Uk;   // [nk][nb][nb] of the tile's k points
  double2* g;          // output of the tile: q stride sgq, k stride nm nb nb
  long sgq;
  long pair0;
  int nk, nm, nb, pad;
};
constexpr int kMaxBandSegs = 32;
struct BandSegs {
  BandSeg s[kMaxBandSegs];
};
cudaError_t launch_band_rotate_multi(const BandSegs& segs, int nseg, long total, int max_nb, int max_nm, int nsm,
                                     cudaStream_t st);
cudaError_t launch_grid_points(int n1, int n2, int n3, const double* shift, double* k, cudaStream_t st);
// E[j][b] = exp(2 pi i (j/N + shift) n(b)), j < N, b < B; slots n(0) = 0, n(2m - 1) = m, n(2m) = -m
cudaError_t launch_axis_phase(int N, int B, double shift, double2* E, cudaStream_t st);
// Wbox[q][box[e]][c] = w_e W[q][e][c]
cudaError_t launch_box_scatter(const double2* W, long sWq, long ldw, int ne, int ncols, const int* box,
                               const double* we, double2* Wbox, long sBq, int nq, cudaStream_t st);
// out[a][j - j0][c] = sum_b E[j][b] in[a][b][c], a < A, c < C, b < B <= 33 (paired: whole unshifted
// axis, B odd)
// out[a][b][r][c] (+)= sum_j conj(E[j0 + j][b]) in[a][j][r][c]  (adjoint of one axis transform)
cudaError_t launch_axis_adj(const double2* in, long sa_in, long sj_in, long ldr_in, int A, int R, int CC, int B,
                            const double2* E, int j0, int nj, double2* out, long sa_out, long sb_out, long ldr_out,
                            int accumulate, cudaStream_t st);
// The same over a whole unshifted axis (j0 = 0, nj = N): the conjugate symmetries of E in j and in
// the slots leave a quarter of the FP64 operations.
cudaError_t launch_axis_adj_paired(const double2* in, long sa_in, long sj_in, long ldr_in, int A, int R, int CC, int B,
                                   const double2* E, int N, double2* out, long sa_out, long sb_out, long ldr_out,
                                   int accumulate, cudaStream_t st);
// G[q][e][c] = w_e Sbox[q][box[e]][c]  (adjoint of the box scatter; we = NULL: weights 1)
cudaError_t launch_box_gather(const double2* Sbox, long sBq, int ncols, const int* box, const double* we, int ne,
                              double2* G, long sGq, int nq, cudaStream_t st);
cudaError_t launch_axis_dft(const double2* in, long sa_in, int A, long C, int B, const double2* E, int N, int j0,
                            int nj, int paired, double2* out, long sa_out, cudaStream_t st);
// The paired transform (whole unshifted axis, j0 = 0, nj = N) in double-float arithmetic on the
// FP32 pipe (~2^-46 of each output's largest term; ~2 FP64 operations per output for the splits
// and joins instead of ~8).  With out32 (C a multiple of nw): the columns c with c mod nw >= nd go
// to out32[a][j][c / nw][c mod nw - nd] as complex64 (a stride sa_out32, rows of nw - nd), rounded
// from the double-float sums without FP64 joins; the others to out as before.
cudaError_t launch_axis_dft_df(const double2* in, long sa_in, int A, long C, int B, const double2* E, int N,
                               double2* out, long sa_out, cudaStream_t st, int nw = 1, int nd = 1,
                               float2* out32 = nullptr, long sa_out32 = 0);

// ---- energy-window prescreening (screen.cu) ------------------------------------------------
// idx[0..*count) = ascending k with some eps[k][n] in [e_lo, e_hi]; flag, pos [nk], tot [ceil(nk/1024)]
cudaError_t launch_window_select(const double* eps, long nk, int nb, double e_lo, double e_hi, int* flag, int* pos,
                                 int* tot, int* idx, int* count, cudaStream_t st);
// flag[i] = 1 if some eps[i][n] lies in [e_lo, e_hi], i < n
cudaError_t launch_window_flags(const double* eps, long n, int nb, double e_lo, double e_hi, int* flag,
                                cudaStream_t st);
// out[j] = kpts[idx[j]] (3 doubles each)
// time-reversal reduction of a uniform grid: kept indices (ascending) and their weights (1 or 2)
cudaError_t launch_ibz_select(int n1, int n2, int n3, const int* t, int* flag, int* pos, int* tot, int* idx,
                              int* count, cudaStream_t st);
cudaError_t launch_ibz_weights(const int* idx, const int* count, int n_max, int n1, int n2, int n3, const int* t,
                               double* w, cudaStream_t st);
cudaError_t launch_gather_points(const double* kpts, const int* idx, int n, double* out, cudaStream_t st);

// ---- fused consumer: electron linewidths from each (q,k) tile without writing g -----------
// part[q][k][n] = pi w_q sum_{m,nu} |g|^2/(2 omega) [(n_B + f) delta(e - e' + omega) + (n_B + 1 - f) delta(e - e' - omega)]
cudaError_t launch_band_linewidth(const double2* Y, long ldy, const double2* Ukq, const double2* Uk, const double* epsk,
                                  const double* epskq, const double* om, const double* wq, int nq, int nk, int nm,
                                  int nb, double kT, double mu, double sigma, double omega_min, double* part,
                                  cudaStream_t st);
// The same terms from g rows already formed ([nu][m][n] per pair, pair stride ldg): any nb, nm.
cudaError_t launch_linewidth_terms(const double2* G, long ldg, const double* epsk, const double* epskq,
                                   const double* om, const double* wq, int nq, int nk, int nm, int nb, double kT,
                                   double mu, double sigma, double omega_min, double* part, cudaStream_t st);
// acc[k][n] += sum_q part[q][k][n]
cudaError_t launch_sum_over_q(const double* part, int nq, long per_q, double* acc, cudaStream_t st);

// ---- adjoint (reverse chain of Eqs. 9-10 for L = sum c |g|^2) ------------------
// In place over the G3 rows of Y: G3bar = V_{k+q} (2 c g) V_k^H with c = w_nk/omega (omega > omega_min);
// Lpair[q*nk + k] = sum c |g|^2 for the pair.  wk: [nk][nb] (tile-local), om: [nq][nm].
cudaError_t launch_band_adjoint(double2* Y, long ldy, const double2* Ukq, const double2* Uk, const double* wk,
                                const double* om, double omega_min, int nq, int nk, int nm, int nb, double* Lpair,
                                cudaStream_t st);
// G3bar = V_{k+q} gbar V_k^H over the pair's G3 row, gbar given ([q][k][nu][m][n], q stride sgq)
cudaError_t launch_band_vjp(double2* Y, long ldy, const double2* gbar, long sgq, const double2* Ukq,
                            const double2* Uk, int nq, int nk, int nm, int nb, cudaStream_t st);
// f[c] = s / invsqrtm[c]^2 (mass of mode index c times s)
cudaError_t launch_mass_factors(const double* invsqrtm, int nm, double s, double* f, cudaStream_t st);
// X[q][c][i] *= f[c], i < blk (in place)
cudaError_t launch_scale_modes(double2* X, int nq, int nm, long blk, const double* f, cudaStream_t st);
// *L += sum_i v[i] (one CTA, fixed order).
cudaError_t launch_sum_into(const double* v, long n, double* L, cudaStream_t st);
// G1bar[q][c][e][b] = sum_nu conj(u[q][c][nu]) G2bar[q][e][nu][b]
cudaError_t launch_mode_rotate_adj(const double2* G2b, const double2* u, int nq, int nm, int ne, int nb2,
                                   double2* G1b, cudaStream_t st);
// Large shapes: L per pair and 2 c g in place over the g rows [nu][m][n] (row stride ldy) of a
// (q batch, k tile); c = wk[k][n] / om[q][nu], 0 for om <= omega_min.
cudaError_t launch_loss_terms(double2* Y, long ldy, const double* wk, const double* om, double omega_min, int nq,
                              int nk, int nm, int nb, double* Lpair, cudaStream_t st);
// g = 0 on the pairs with keep[q nk + k] == 0 (pair (q, k): per elements of eb = 8 or 16 bytes at
// element q sgq + k per).
cudaError_t launch_zero_masked(void* g, int eb, long sgq, long per, int nq, int nk, const int* keep, cudaStream_t st);
// out[b] = in[b]^H for a batch of n x n complex matrices.
cudaError_t launch_conj_transpose(const double2* in, int n, long batch, double2* out, cudaStream_t st);

// ---- mixed form (split-TF32 tensor-core Re->k contraction) -------------------------
// TMA descriptor (CUtensorMap, 128 bytes) over a row-major FP32 [rows][kp] array:
// box 32 (k) x box_rows, 128-byte swizzle.  kp must be a multiple of 32.
cudaError_t make_tc_map(void* map_out, const float* base, long rows, int kp, int box_rows);
// C[q][m][n] = (Ahi Bhi + Ahi Blo + Alo Bhi) over k; A rows a_row0 + m (box 128 rows),
// B rows q*Nr + n (box 256 rows); C row stride ldc, batch stride sC; err |= timeout bits.
cudaError_t launch_tc_split_gemm(const void* mAhi, const void* mAlo, const void* mBhi, const void* mBlo, int M,
                                 int a_row0, int Nr, int Kp, int nq, float* C, long ldc, long sC, int* err,
                                 cudaStream_t st);
cudaError_t launch_split_a(const double2* P, long ldp, int n, int ne, int kp, float* Ahi, float* Alo,
                           cudaStream_t st);
cudaError_t launch_split_b(const double2* W, long ldw, long sW, int col0, int ncols, int ne, int kp, int nq,
                           float* Bhi, float* Blo, cudaStream_t st);
// Band rotation with double-float accumulation (FP64 gauges as float pairs), complex64 out.
cudaError_t launch_band_rotate_ff(const float* Y, long ldy_floats, const double2* Ukq, const double2* Uk, int nq,
                                  int nk, int nm, int nb, float* g, long sgq_floats, cudaStream_t st, const int* keep = nullptr);
// the same from complex128 G3 rows (product-grid path of the mixed form); g complex64, sgq in elements
cudaError_t launch_band_rotate_ff_f64(const double2* Y, long ldy, const double2* Ukq, const double2* Uk, int nq, int nk,
                                      int nm, int nb, float2* g, long sgq, cudaStream_t st, const int* keep = nullptr);
// Fixed-point BF16 digits (A: 3, B: 4 per value; exact tensor-core accumulation); D slices of n*kp / slice.
cudaError_t make_tc_map_bf16(void* map_out, const void* base, long rows, int kp, int box_rows);
cudaError_t launch_digits_a(const double2* P, long ldp, int n, int ne, int kp, double scale, int ndig, void* D,
                            cudaStream_t st, int plane_rows = 0);
// complex64 as float pairs -> complex128
cudaError_t launch_f32pairs_to_c128(const float2* X, long n, double2* Y, cudaStream_t st);
cudaError_t launch_digits_b(const double2* W, long ldw, long sW, int col0, int ncols, int ne, int kp, int nq,
                            float* sB, void* D, long slice, int ndig, cudaStream_t st);
// complex128 H[i] = (hi + lo of real output 2i, hi + lo of 2i + 1), i < n
cudaError_t launch_pairs_to_c128(const float2* Hp, long n, double2* H, cudaStream_t st);
// C = sA sB[col] 2^-16 sum_l 2^-8l L_l on tcgen05 kind::f16; maps: 3 CUtensorMaps (A), 4 (B).
// 2-D BF16 tensor map, box 32 x box_rows, 64-byte swizzle (operands of the H(k+q) kernel)
cudaError_t make_tc_map_bf16_sw64(void* map_out, const void* base, long rows, int kp, int box_rows);
// H(k+q) on the tensor cores from 5 x 5 BF16 digits: C[q][m][n] = (hi, lo) float pairs, ldc/sC in float2
cudaError_t launch_tc_hkq_gemm(const void* maps_a5, const void* maps_b5, int M, int a_row0, int Nr, int Kp, int nq,
                               float sA, const float* sB, float2* C, long ldc, long sC, int* err, cudaStream_t st);
// Same product batched over q with A rows a_row0 + ((q + a_qoff) mod a_mod) a_stride + m; morder = 1
// takes the m tiles fastest (M of a few tiles sharing each B tile); ndig = 4 or 5 digits per
// operand (the first ndig maps of each array are read).
cudaError_t launch_tc_hkq_gemm_b(const void* maps_a5, const void* maps_b5, int M, int a_row0, int Nr, int Kp, int nq,
                                 float sA, const float* sB, float2* C, long ldc, long sC, int* err, int a_mod,
                                 int a_qoff, int a_stride, int morder, int ndig, cudaStream_t st);
cudaError_t launch_tc_fixed_gemm(const void* maps_a3, const void* maps_b4, int M, int a_row0, int Nr, int Kp, int nq,
                                 float sA, const float* sB, float* C, long ldc, long sC, int* err, cudaStream_t st);
// Batched products of the band rotation: four digits per operand (maps: 4 CUtensorMaps each,
// 64-byte swizzle), levels <= 3 in two accumulators (level 0 exact), two accumulator sets so the
// epilogue overlaps the next tile; C one FP32 per element (ldc, sC in floats); A rows as
// launch_tc_hkq_gemm_b, m tiles fastest.
cudaError_t launch_tc_band_gemm(const void* maps_a4, const void* maps_b4, int M, int a_row0, int Nr, int Kp, int nq,
                                float sA, const float* sB, float* C, long ldc, long sC, int* err, int a_mod,
                                int a_qoff, int a_stride, cudaStream_t st);
// Band rotation of large shapes on the tensor cores (mixed form): g[iq][kk] (complex64, rows iq
// sgq apart, pair (iq, kk) at kk nm nb^2) = V_{k+q}^H G3_nu V_k for the nq x nk pairs of a tile,
// G3 at Y + (iq nk + kk) ldy + y_off (complex128, or complex64 when y_f32; ldy, y_off in complex
// elements), V_{k+q} at Ukq + (iq nk + kk) nb^2, V_k at Uk + kk nb^2.
// work: at least band_tc_work_bytes(nk, nm, nb, 1) bytes; more lets more pairs go per chunk.
size_t band_tc_work_bytes(int nk, int nm, int nb, long pairs);
bool band_tc_supported(int nm, int nb);
// Fused tensor-core band rotation for nb <= 16, nm nb <= 128 (complex64 g, ~2^-31 relative to each
// pair's largest element): Y rows of G3 per pair (complex128 or, y_f32, complex64), ldy complex
// elements apart; keep (optional) zeroes screened pairs; *err |= 16 on a barrier timeout.
bool band_tc_small_supported(int nm, int nb);
cudaError_t launch_band_tc_small(const void* Y, int y_f32, long ldy, const double2* Ukq, const double2* Uk, int nq,
                                 int nk, int nm, int nb, float2* g, long sgq, const int* keep, int* err,
                                 cudaStream_t st);
// The same rotation at FP64 accuracy (six-digit operands, exact level sums, integer assembly of
// the doubles): complex128 G3 in, complex128 g out, ~5e-14 of each pair's largest element.
cudaError_t launch_band_tc_small64(const double2* Y, long ldy, const double2* Ukq, const double2* Uk, int nq, int nk,
                                   int nm, int nb, double2* g, long sgq, const int* keep, int* err, cudaStream_t st);
// General form: pair (iq, kk) reads X + iq xq + kk xk and writes out + iq oq + kk ok (may be the
// same rows); adj: V_{k+q} X V_k^H instead of V_{k+q}^H X V_k; wk non-NULL: the adjoint's loss
// terms, Lpair[iq nk + kk] = sum c |g|^2 and 2 c g written (c = wk[kk][n] / om[iq][nu], 0 for
// om <= omega_min).
cudaError_t launch_band_tc_small64_ex(const double2* X, long xq, long xk, const double2* Ukq, const double2* Uk, int nq,
                                      int nk, int nm, int nb, double2* out, long oq, long ok, const int* keep, bool adj,
                                      const double* wk, const double* om, double omega_min, double* Lpair, int* err,
                                      cudaStream_t st);
// FP64-accuracy complex GEMM on the tensor cores (seven base-128 digits per operand, exact level
// sums, doubles assembled from 64-bit integers): digit planes [7][rows][Kp] (bf16) of a complex
// P with element (r, e) at P[r sr + e se] (K = (e, re/im), Kp a multiple of 32, 2 ne <= Kp), with
// the largest biased exponent of each row in ea; of the columns of W[q][e][c] (nq x ncol columns;
// conj(W) with cj) as 2 ncol rows per q (Re / Im of the product), with the column exponents in eb
// (per row).
cudaError_t launch_zdigits_rows(const double2* P, long sr, long se, int rows, int ne, int Kp, int* ea, void* planes,
                                cudaStream_t st);
cudaError_t launch_zdigits_cols(const double2* W, long ldw, long sW, int nq, int ne, int ncol, int Kp, int cj, int* eb,
                                void* planes, cudaStream_t st);
// C[q sCq + row ldc + c scol] (=, or += with acc) sum_e P[a_row0 + row][e] W[q][e][c] for rows < M
// and the N = nq ncq real columns (ncq = 2 ncol per q; C complex128); Kp <= 512.  *err |= 1..8 on
// a barrier timeout.
cudaError_t launch_tc_zgemm64(const void* a_planes, long a_rows, int a_row0, int M, const int* ea, const void* b_planes,
                              int N, const int* eb, int Kp, double2* C, int ncq, long ldc, long sCq, long scol, int acc,
                              int* err, cudaStream_t st);
cudaError_t launch_band_tc(const void* Y, int y_f32, long ldy, long y_off, const double2* Ukq, const double2* Uk, int nq,
                           int nk, int nm, int nb, float2* g, long sgq, void* work, size_t work_bytes, int* err,
                           cudaStream_t st);

}  // namespace eph
