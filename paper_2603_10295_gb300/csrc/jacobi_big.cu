// Batched Hermitian eigensolver for 16 < n <= 256 (the band Hamiltonians H(k), H(k+q) and
// the dynamical matrices D(q) of Eqs. 4-5 when Nb or 3 Na exceed a warp's register file):
// one CTA per matrix.
//
// Two solvers share the FP64 rotation round of the cyclic parallel Jacobi method:
//   - k_jacobi_big: plain FP64 sweeps on a global-memory working copy (the reference form);
//   - the preconditioned form (launch_eigh_big): FP32 sweeps on a packed copy held in shared
//     memory, two FP64 Newton-Schulz re-orthonormalisations of the FP32 eigenvectors and
//     A' = V^H A V as batched FP64 GEMMs, then FP64 sweeps on A' until every remaining
//     rotation angle is small enough for a first-order finish.  The FP64 pipe, which bounds
//     the plain form at about eleven sweeps per matrix, then carries ~one sweep and seven
//     n^3 products; the FP32 sweeps run at FP32 rate from shared memory.
#include "eph_kernels.cuh"

namespace eph {

namespace {

// Circle (round-robin) schedule over np (even) indices: in round r of a sweep, pair 0 couples
// r with np - 1 and pair i > 0 couples (r + i) mod (np - 1) with (r - i) mod (np - 1); the
// np/2 pairs of a round are disjoint and every unordered pair meets once in np - 1 rounds.
__device__ __forceinline__ void circle_pair(int i, int r, int np, int& p, int& q) {
  const int m = np - 1;
  if (i == 0) {
    p = r;
    q = m;
  } else {
    p = (r + i) % m;
    q = (r - i + m) % m;
  }
  if (p > q) {
    const int t = p;
    p = q;
    q = t;
  }
}

template <typename T>
__device__ T block_sum(T x, T* red) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  const int tid = threadIdx.x, nt = blockDim.x;
  if ((tid & 31) == 0) red[tid >> 5] = x;
  __syncthreads();
  T t = 0;
  for (int i = 0; i < (nt >> 5); ++i) t += red[i];
  __syncthreads();
  return t;
}

// Rotation of the pair (p, q): with b = A_pq, d = A_qq - A_pp and r = 2 sgn(d) / (|d| + sqrt(d^2 + 4|b|^2))
// (the smaller root of the angle equation), c = 1 / sqrt(1 + r^2 |b|^2) and sigma = c r b, the unitary
//   J = [[c, sigma], [-conj(sigma), c]]  (rows and columns p, q)
// makes (J^H A J)_pq = 0 with diagonal A_pp - r|b|^2, A_qq + r|b|^2.  Columns mix as
// col_p' = c col_p - conj(sigma) col_q, col_q' = sigma col_p + c col_q; rows (J^H) as
// row_p' = c row_p - sigma row_q, row_q' = conj(sigma) row_p + c row_q.
struct Round64 {
  int sp[128], sq[128], son[128];
  double sc[128], stb[128], sapp[128], saqq[128];
  double2 ssg[128];
};

// One round of FP64 rotations on M (n x n, row-major, global) accumulating V <- V J.
// Threshold form: a pair is rotated only if |A_pq|^2 > max(thresh2, th2 (A_qq - A_pp)^2), i.e.
// if its angle is above sqrt(th2) (th2 = 0: every pair above thresh2); the rest is left to
// the first-order finish.
__device__ void fp64_round(double2* __restrict__ M, double2* __restrict__ U, int n, int np, int r, double thresh2,
                           double th2, Round64& s) {
  // (thresh2 also carries the rounding-level coupling that the polish accepts without rotation)
  const int tid = threadIdx.x, nt = blockDim.x, npairs = np / 2;
  for (int i = tid; i < npairs; i += nt) {
    int p, q;
    circle_pair(i, r, np, p, q);
    double c = 1.0, tb = 0.0;
    double2 sig = make_double2(0.0, 0.0);
    double app = 0.0, aqq = 0.0;
    int on = 0;
    if (q < n) {
      app = M[(long)p * n + p].x;
      aqq = M[(long)q * n + q].x;
      const double2 b = M[(long)p * n + q];
      const double b2 = fma(b.x, b.x, b.y * b.y);
      const double dd = aqq - app;
      if (b2 > thresh2 && b2 > th2 * (dd * dd)) {
        on = 1;
        const double rr = copysign(2.0, dd) / (fabs(dd) + sqrt(fma(dd, dd, 4.0 * b2)));
        tb = rr * b2;
        c = rsqrt(fma(rr * rr, b2, 1.0));
        sig = make_double2(c * rr * b.x, c * rr * b.y);
      }
    }
    s.sp[i] = p;
    s.sq[i] = q;
    s.son[i] = on;
    s.sc[i] = c;
    s.ssg[i] = sig;
    s.stb[i] = tb;
    s.sapp[i] = app;
    s.saqq[i] = aqq;
  }
  __syncthreads();
  // columns of A and V
  for (long idx = tid; idx < (long)npairs * n; idx += nt) {
    const int x = (int)(idx / npairs), i = (int)(idx - (long)x * npairs);
    if (!s.son[i]) continue;
    const int p = s.sp[i], q = s.sq[i];
    const double c = s.sc[i];
    const double2 g = s.ssg[i];
    double2* rowA = M + (long)x * n;
    double2* rowU = U + (long)x * n;
    const double2 ap = rowA[p], aq = rowA[q], up = rowU[p], uq = rowU[q];
    rowA[p] = make_double2(fma(c, ap.x, -fma(g.x, aq.x, g.y * aq.y)), fma(c, ap.y, -fma(g.x, aq.y, -g.y * aq.x)));
    rowA[q] = make_double2(fma(c, aq.x, fma(g.x, ap.x, -g.y * ap.y)), fma(c, aq.y, fma(g.x, ap.y, g.y * ap.x)));
    rowU[p] = make_double2(fma(c, up.x, -fma(g.x, uq.x, g.y * uq.y)), fma(c, up.y, -fma(g.x, uq.y, -g.y * uq.x)));
    rowU[q] = make_double2(fma(c, uq.x, fma(g.x, up.x, -g.y * up.y)), fma(c, uq.y, fma(g.x, up.y, g.y * up.x)));
  }
  __syncthreads();
  // rows of A
  for (long idx = tid; idx < (long)npairs * n; idx += nt) {
    const int i = (int)(idx / n), y = (int)(idx - (long)i * n);
    if (!s.son[i]) continue;
    const int p = s.sp[i], q = s.sq[i];
    const double c = s.sc[i];
    const double2 g = s.ssg[i];
    double2* a = M + (long)p * n + y;
    double2* b = M + (long)q * n + y;
    const double2 xl = *a, xh = *b;
    *a = make_double2(fma(c, xl.x, -fma(g.x, xh.x, -g.y * xh.y)), fma(c, xl.y, -fma(g.x, xh.y, g.y * xh.x)));
    *b = make_double2(fma(c, xh.x, fma(g.x, xl.x, g.y * xl.y)), fma(c, xh.y, fma(g.x, xl.y, -g.y * xl.x)));
  }
  __syncthreads();
  // exact values of each rotated 2x2 block
  for (int i = tid; i < npairs; i += nt) {
    if (!s.son[i]) continue;
    const int p = s.sp[i], q = s.sq[i];
    M[(long)p * n + q] = make_double2(0.0, 0.0);
    M[(long)q * n + p] = make_double2(0.0, 0.0);
    M[(long)p * n + p] = make_double2(s.sapp[i] - s.stb[i], 0.0);
    M[(long)q * n + q] = make_double2(s.saqq[i] + s.stb[i], 0.0);
  }
  __syncthreads();
}

// ascending order, ties by index: rank[j] = #{i : l_i < l_j or (l_i == l_j and i < j)}
__device__ __forceinline__ int sort_rank(const double* lam, int n, int j) {
  const double l = lam[j];
  int rank = 0;
  for (int i = 0; i < n; ++i) {
    const double li = lam[i];
    if (li < l || (li == l && i < j)) ++rank;
  }
  return rank;
}

int threads_for(long work) {
  int t = (int)(((work + 31) / 32) * 32);
  return t < 128 ? 128 : (t > 1024 ? 1024 : t);
}

}  // namespace

// ----------------------------------------------------------------------------
// Plain FP64 form: sweeps on a global working copy until the off-diagonal norm falls
// below 1e-15 ||A||_F, then one more sweep (cap max_sweeps -> *status |= 1).
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_jacobi_big(const double2* __restrict__ A, long sA, long lda, int n,
                                                    double* __restrict__ w, long sw, double2* __restrict__ V, long sV,
                                                    double2* __restrict__ work, int max_sweeps,
                                                    int* __restrict__ status) {
  __shared__ Round64 rs;
  __shared__ double red[32];
  __shared__ double slam[256];
  __shared__ int srank[256];
  const long mat = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  const long nn = (long)n * n;
  double2* M = work + mat * nn;  // working copy, row-major
  double2* U = V + mat * sV;     // accumulated eigenvectors, row-major (columns)
  const double2* Ain = A + mat * sA;
  for (long i = tid; i < nn; i += nt) {
    const int r = (int)(i / n), c = (int)(i - (long)r * n);
    double2 v = Ain[(long)r * lda + c];
    if (r == c) v.y = 0.0;
    M[i] = v;
    U[i] = make_double2(r == c ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  double part = 0.0;
  for (long i = tid; i < nn; i += nt) part = fma(M[i].x, M[i].x, fma(M[i].y, M[i].y, part));
  const double fro2 = block_sum(part, red);
  const double thresh2 = 1e-36 * fro2 + 1e-300;
  const double tol2 = 1e-30 * fro2;
  const int np = (n + 1) & ~1;
  bool conv = false;
  int post = 0, sweep = 0;
  while (!(conv && post >= 1) && sweep < max_sweeps) {
    for (int r = 0; r < np - 1; ++r) fp64_round(M, U, n, np, r, thresh2, 0.0, rs);
    ++sweep;
    if (conv) ++post;
    part = 0.0;
    for (long i = tid; i < nn; i += nt) {
      const int r = (int)(i / n), c = (int)(i - (long)r * n);
      if (r != c) part = fma(M[i].x, M[i].x, fma(M[i].y, M[i].y, part));
    }
    if (block_sum(part, red) <= tol2) conv = true;
  }
  if (tid == 0 && !conv) atomicOr(status, 1);
  for (int j = tid; j < n; j += nt) slam[j] = M[(long)j * n + j].x;
  __syncthreads();
  for (int j = tid; j < n; j += nt) {
    const int rank = sort_rank(slam, n, j);
    w[mat * sw + rank] = slam[j];
    srank[j] = rank;
  }
  __syncthreads();
  for (long i = tid; i < nn; i += nt) M[i] = U[i];
  __syncthreads();
  for (long i = tid; i < nn; i += nt) {
    const int r = (int)(i / n), j = (int)(i - (long)r * n);
    U[(long)r * n + srank[j]] = M[i];
  }
}

cudaError_t launch_jacobi_big(const double2* A, long sA, long lda, int n, long batch, double* w, long sw, double2* V,
                              long sV, double2* work, int max_sweeps, int* status, cudaStream_t st) {
  if (batch <= 0) return cudaSuccess;
  if (n < 1 || n > 256 || sV != (long)n * n) return cudaErrorInvalidValue;
  if (batch > 2147483647L) return cudaErrorInvalidConfiguration;
  // a round's column and row mixes touch n^2 / 2 elements each; with few matrices per SM the
  // latency of these global (L2-resident) accesses needs many threads in flight: about n^2 / 8
  // threads (128 .. 1024)
  k_jacobi_big<<<(unsigned)batch, threads_for((long)n * n / 8), 0, st>>>(A, sA, lda, n, w, sw, V, sV, work,
                                                                         max_sweeps, status), note_launch();
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Preconditioned form.
// ----------------------------------------------------------------------------
namespace {

// Packed Hermitian matrix in shared memory (np x np floats, row stride lds): for x < y,
// S[x][y] = Re A_xy and S[y][x] = Im A_xy; S[x][x] = A_xx.
__device__ __forceinline__ float2 hget(const float* S, int lds, int x, int y) {
  return x < y ? make_float2(S[x * lds + y], S[y * lds + x]) : make_float2(S[y * lds + x], -S[x * lds + y]);
}
__device__ __forceinline__ void hset(float* S, int lds, int x, int y, float2 v) {
  if (x < y) {
    S[x * lds + y] = v.x;
    S[y * lds + x] = v.y;
  } else {
    S[y * lds + x] = v.x;
    S[x * lds + y] = -v.y;
  }
}
// column mix (A J): c a - conj(s) b and s a + c b
__device__ __forceinline__ float2 col_lo(float c, float2 s, float2 a, float2 b) {
  return make_float2(fmaf(c, a.x, -fmaf(s.x, b.x, s.y * b.y)), fmaf(c, a.y, -fmaf(s.x, b.y, -s.y * b.x)));
}
__device__ __forceinline__ float2 col_hi(float c, float2 s, float2 a, float2 b) {
  return make_float2(fmaf(c, b.x, fmaf(s.x, a.x, -s.y * a.y)), fmaf(c, b.y, fmaf(s.x, a.y, s.y * a.x)));
}
// row mix (J^H A): c a - s b and conj(s) a + c b
__device__ __forceinline__ float2 row_lo(float c, float2 s, float2 a, float2 b) {
  return make_float2(fmaf(c, a.x, -fmaf(s.x, b.x, -s.y * b.y)), fmaf(c, a.y, -fmaf(s.x, b.y, s.y * b.x)));
}
__device__ __forceinline__ float2 row_hi(float c, float2 s, float2 a, float2 b) {
  return make_float2(fmaf(c, b.x, fmaf(s.x, a.x, s.y * a.y)), fmaf(c, b.y, fmaf(s.x, a.y, -s.y * a.x)));
}

}  // namespace

// FP32 sweeps on the packed copy (n padded to even np with a zero row and column, which no
// rotation touches) until the off-diagonal norm is below 1e-6 ||A||_F or max_sweeps; the FP32
// eigenvectors (in shared memory when they fit, else at vglob) are written as FP64 to Vout.
// A round is one pass over the off-diagonal 2x2 blocks (I, J), I < J, of the round's pairs:
// B' = J_I^H B J_J (each block read and written by one thread), plus the exact diagonal blocks.
__global__ void __launch_bounds__(1024) k_jacobi32_big(const double2* __restrict__ A, long sA, long lda, int n, int np,
                                                      int lds, int vsm, float2* __restrict__ vglob,
                                                      double2* __restrict__ Vout, int max_sweeps) {
  extern __shared__ __align__(16) float s32[];
  __shared__ int sp[128], sq[128], son[128];
  __shared__ float sc[128], sd0[128], sd1[128];
  __shared__ float2 ssg[128];
  __shared__ double redd[32];
  __shared__ float redf[32];
  const long mat = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x, npairs = np / 2;
  float* S = s32;
  float2* Vf = vsm ? reinterpret_cast<float2*>(s32 + (((long)np * lds + 3) & ~3L)) : vglob + mat * (long)np * np;
  const double2* Ain = A + mat * sA;
  double part = 0.0;
  for (int idx = tid; idx < np * np; idx += nt) {
    const int r = idx / np, c = idx - r * np;
    if (r <= c) {
      const double2 a = (r < n && c < n) ? Ain[(long)r * lda + c] : make_double2(0.0, 0.0);
      if (r == c) {
        S[r * lds + r] = (float)a.x;
        part = fma(a.x, a.x, part);
      } else {
        S[r * lds + c] = (float)a.x;
        S[c * lds + r] = (float)a.y;
        part += 2.0 * fma(a.x, a.x, a.y * a.y);
      }
    }
    Vf[idx] = make_float2(r == c ? 1.f : 0.f, 0.f);
  }
  const double fro2 = block_sum(part, redd);  // (its barriers also publish S and Vf)
  // rotations below |A_pq| = 1e-9 ||A||_F are skipped: FP32 sweeps cannot resolve them
  const float thr = (float)(1e-18 * fro2);
  const float tol = (float)(1e-12 * fro2);
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    for (int r = 0; r < np - 1; ++r) {
      for (int i = tid; i < npairs; i += nt) {
        int p, q;
        circle_pair(i, r, np, p, q);
        const float app = S[p * lds + p], aqq = S[q * lds + q];
        const float bx = S[p * lds + q], by = S[q * lds + p];
        const float b2 = fmaf(bx, bx, by * by);
        float c = 1.f, tb = 0.f;
        float2 g = make_float2(0.f, 0.f);
        int on = 0;
        if (b2 > thr) {
          const float dd = aqq - app;
          const float rr = copysignf(2.f, dd) / (fabsf(dd) + sqrtf(fmaf(dd, dd, 4.f * b2)));
          tb = rr * b2;
          c = rsqrtf(fmaf(rr * rr, b2, 1.f));
          g = make_float2(c * rr * bx, c * rr * by);
          on = 1;
        }
        sp[i] = p;
        sq[i] = q;
        sc[i] = c;
        ssg[i] = g;
        sd0[i] = app - tb;
        sd1[i] = aqq + tb;
        son[i] = on;
      }
      __syncthreads();
      // off-diagonal blocks
      for (int t = tid; t < npairs * npairs; t += nt) {
        const int I = t / npairs, J = t - I * npairs;
        if (I >= J || !(son[I] | son[J])) continue;
        const int p = sp[I], q = sq[I], u = sp[J], v = sq[J];
        const float c1 = sc[I], c2 = sc[J];
        const float2 g1 = ssg[I], g2 = ssg[J];
        const float2 b00 = hget(S, lds, p, u), b01 = hget(S, lds, p, v);
        const float2 b10 = hget(S, lds, q, u), b11 = hget(S, lds, q, v);
        const float2 t00 = col_lo(c2, g2, b00, b01), t01 = col_hi(c2, g2, b00, b01);
        const float2 t10 = col_lo(c2, g2, b10, b11), t11 = col_hi(c2, g2, b10, b11);
        hset(S, lds, p, u, row_lo(c1, g1, t00, t10));
        hset(S, lds, q, u, row_hi(c1, g1, t00, t10));
        hset(S, lds, p, v, row_lo(c1, g1, t01, t11));
        hset(S, lds, q, v, row_hi(c1, g1, t01, t11));
      }
      // diagonal blocks
      for (int i = tid; i < npairs; i += nt) {
        if (!son[i]) continue;
        const int p = sp[i], q = sq[i];
        S[p * lds + p] = sd0[i];
        S[q * lds + q] = sd1[i];
        S[p * lds + q] = 0.f;
        S[q * lds + p] = 0.f;
      }
      // eigenvector columns
      for (int t = tid; t < np * npairs; t += nt) {
        const int x = t / npairs, i = t - x * npairs;
        if (!son[i]) continue;
        const int p = sp[i], q = sq[i];
        float2* row = Vf + (long)x * np;
        const float2 vp = row[p], vq = row[q];
        row[p] = col_lo(sc[i], ssg[i], vp, vq);
        row[q] = col_hi(sc[i], ssg[i], vp, vq);
      }
      __syncthreads();
    }
    float off = 0.f;
    for (int idx = tid; idx < np * np; idx += nt) {
      const int r = idx / np, c = idx - r * np;
      if (r != c) {
        const float x = S[r * lds + c];
        off = fmaf(x, x, off);
      }
    }
    if (2.f * block_sum(off, redf) <= tol) break;
  }
  double2* Vo = Vout + mat * (long)n * n;
  for (int idx = tid; idx < n * n; idx += nt) {
    const int r = idx / n, c = idx - r * n;
    const float2 v = Vf[(long)r * np + c];
    Vo[idx] = make_double2((double)v.x, (double)v.y);
  }
}

// Newton-Schulz step V <- V (3I - V^H V) / 2 = 1.5 V - 0.5 T with T = V (V^H V).
__global__ void k_ns_update(double2* __restrict__ V, const double2* __restrict__ T, long total) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const double2 v = V[i], t = T[i];
  V[i] = make_double2(fma(1.5, v.x, -0.5 * t.x), fma(1.5, v.y, -0.5 * t.y));
}

// FP64 threshold sweeps on A' = V^H A V (Mw, its Hermitian part taken first; only pairs whose
// angle is above sqrt(th2) and whose coupling is above polish_tol ||A||_F are rotated),
// accumulating into U, until every remaining coupling has an angle |A'_ij / (A'_jj - A'_ii)|^2
// below th2 or is below polish_tol ||A||_F (tested before the first sweep when try_before), or
// the off-diagonal norm is below polish_tol ||A||_F.  On the angle exit the
// first-order finish is prepared: Mw becomes X with X_ij = A'_ij / (A'_jj - A'_ii) (zero diagonal),
// so that V = U (I + X) completes the eigenvectors to th2 (the update is anti-Hermitian to first
// order), and lam_j = A'_jj + sum_i |A'_ij|^2 / (A'_jj - A'_ii) the eigenvalues; otherwise X = 0.
__global__ void __launch_bounds__(1024) k_jacobi_polish_big(double2* __restrict__ Mw, double2* __restrict__ Uw, int n,
                                                           double* __restrict__ lamw, double polish_tol, double th2,
                                                           int try_before, int max_sweeps, int* __restrict__ status) {
  __shared__ Round64 rs;
  __shared__ double red[32];
  __shared__ double slam[256];
  const long mat = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  const long nn = (long)n * n;
  double2* M = Mw + mat * nn;
  double2* U = Uw + mat * nn;
  double part = 0.0;
  for (long idx = tid; idx < nn; idx += nt) {
    const int r = (int)(idx / n), c = (int)(idx - (long)r * n);
    if (r < c) {
      const double2 a = M[idx], b = M[(long)c * n + r];
      const double2 h = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
      M[idx] = h;
      M[(long)c * n + r] = make_double2(h.x, -h.y);
      part += 2.0 * fma(h.x, h.x, h.y * h.y);
    } else if (r == c) {
      const double d = M[idx].x;
      M[idx] = make_double2(d, 0.0);
      part = fma(d, d, part);
    }
  }
  const double fro2 = block_sum(part, red);
  const double thresh2 = 1e-36 * fro2 + 1e-300;
  const double tol2 = polish_tol * polish_tol * fro2;
  const int np = (n + 1) & ~1;
  bool conv = false, fin = false;
  int sweep = 0;
  for (;;) {
    if (sweep > 0 || try_before) {
      int bad = 0;
      for (long idx = tid; idx < nn; idx += nt) {
        const int r = (int)(idx / n), c = (int)(idx - (long)r * n);
        if (r < c) {
          const double2 m = M[idx];
          const double gap = M[(long)c * n + c].x - M[(long)r * n + r].x;
          const double m2 = fma(m.x, m.x, m.y * m.y);
          // a small angle (first-order finish) or a coupling at the polish tolerance
          if (!(m2 <= th2 * (gap * gap)) && !(m2 <= tol2)) bad = 1;
        }
      }
      if (!__syncthreads_or(bad)) {
        fin = true;
        break;
      }
    }
    if (conv || sweep >= max_sweeps) break;
    for (int r = 0; r < np - 1; ++r) fp64_round(M, U, n, np, r, thresh2 > tol2 ? thresh2 : tol2, th2, rs);
    ++sweep;
    part = 0.0;
    for (long idx = tid; idx < nn; idx += nt) {
      const int r = (int)(idx / n), c = (int)(idx - (long)r * n);
      if (r != c) part = fma(M[idx].x, M[idx].x, fma(M[idx].y, M[idx].y, part));
    }
    if (block_sum(part, red) <= tol2) conv = true;
  }
  if (tid == 0 && !(conv || fin)) atomicOr(status, 1);
  for (int j = tid; j < n; j += nt) {
    const double lj = M[(long)j * n + j].x;
    double dl = 0.0;
    if (fin) {
      for (int i = 0; i < n; ++i) {
        const double2 m = M[(long)i * n + j];
        const double gap = lj - M[(long)i * n + i].x, m2 = fma(m.x, m.x, m.y * m.y);
        if (i != j && m2 != 0.0 && m2 <= th2 * (gap * gap)) dl += m2 / gap;
      }
    }
    slam[j] = lj + dl;
  }
  __syncthreads();
  for (long idx = tid; idx < nn; idx += nt) {
    const int i = (int)(idx / n), j = (int)(idx - (long)i * n);
    if (i == j) continue;
    const double2 m = M[idx];
    double2 x = make_double2(0.0, 0.0);
    const double gap = M[(long)j * n + j].x - M[(long)i * n + i].x, m2 = fma(m.x, m.x, m.y * m.y);
    if (fin && m2 != 0.0 && m2 <= th2 * (gap * gap)) {  // couplings left at tolerance level stay unrotated
      const double inv = 1.0 / gap;
      x = make_double2(m.x * inv, m.y * inv);
    }
    M[idx] = x;
  }
  __syncthreads();
  for (int j = tid; j < n; j += nt) {
    M[(long)j * n + j] = make_double2(0.0, 0.0);
    lamw[mat * n + j] = slam[j];
  }
}

// V[:, rank_j] = U[:, j] + T[:, j] (T = U X), w[rank_j] = lam_j, ascending with ties by index.
__global__ void k_eig_sort_big(const double2* __restrict__ Uw, const double2* __restrict__ Tw,
                               const double* __restrict__ lamw, int n, double* __restrict__ w, long sw,
                               double2* __restrict__ V, long sV) {
  __shared__ double slam[256];
  __shared__ int srank[256];
  const long mat = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  const long nn = (long)n * n;
  for (int j = tid; j < n; j += nt) slam[j] = lamw[mat * n + j];
  __syncthreads();
  for (int j = tid; j < n; j += nt) {
    const int rank = sort_rank(slam, n, j);
    srank[j] = rank;
    w[mat * sw + rank] = slam[j];
  }
  __syncthreads();
  const double2* U = Uw + mat * nn;
  const double2* T = Tw + mat * nn;
  double2* out = V + mat * sV;
  for (long idx = tid; idx < nn; idx += nt) {
    const int r = (int)(idx / n), j = (int)(idx - (long)r * n);
    const double2 u = U[idx], t = T[idx];
    out[(long)r * n + srank[j]] = make_double2(u.x + t.x, u.y + t.y);
  }
}

namespace {

struct Eigh32Shape {
  int np, lds, vsm;
  size_t smem;
};

// shared-memory plan of k_jacobi32_big; false when the packed matrix does not fit
bool eigh32_shape(int n, Eigh32Shape& s) {
  static int optin = -1, static_smem = 0;
  if (optin < 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return false;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_jacobi32_big) != cudaSuccess) return false;
    static_smem = (int)fa.sharedSizeBytes;
  }
  s.np = (n + 1) & ~1;
  s.lds = s.np + 1;
  const size_t packed = (((size_t)s.np * s.lds + 3) & ~(size_t)3) * sizeof(float);
  const size_t vbytes = (size_t)s.np * s.np * sizeof(float2);
  const size_t avail = (size_t)(optin - static_smem);
  if (packed > avail) return false;
  s.vsm = packed + vbytes <= avail;
  s.smem = packed + (s.vsm ? vbytes : 0);
  return true;
}

}  // namespace

bool eigh_big_supported(int n) {
  Eigh32Shape s;
  return n > 16 && n <= 256 && eigh32_shape(n, s);
}

size_t eigh_big_work_bytes(int n, long batch) {
  return (size_t)batch * n * n * sizeof(double2) * 4 + (size_t)batch * n * sizeof(double);
}

cudaError_t launch_eigh_big(const double2* A, long sA, long lda, int n, long batch, double* w, long sw, double2* V,
                            long sV, void* work, double polish_tol, int max_sweeps, int* status, cudaStream_t st) {
  if (batch <= 0) return cudaSuccess;
  Eigh32Shape sh;
  if (n <= 16 || n > 256 || sV != (long)n * n || !eigh32_shape(n, sh)) return cudaErrorInvalidValue;
  const long nn = (long)n * n;
  const long CH = 65535;  // batched-GEMM grid limit
  for (long b0 = 0; b0 < batch; b0 += CH) {
    const int nb = (int)(batch - b0 < CH ? batch - b0 : CH);
    const double2* Ab = A + b0 * sA;
    double2* M = static_cast<double2*>(work);
    double2* Vw = M + (long)nb * nn;
    double2* G = Vw + (long)nb * nn;
    double2* T = G + (long)nb * nn;
    double* lam = reinterpret_cast<double*>(T + (long)nb * nn);
    cudaError_t e;
    if (sh.smem > 48 * 1024) {
      e = cudaFuncSetAttribute(k_jacobi32_big, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem);
      if (e != cudaSuccess) return e;
    }
    // FP32 eigenvectors; when they do not fit in shared memory they live in G (free until the Gram)
    k_jacobi32_big<<<(unsigned)nb, threads_for((long)sh.np * sh.np / 4), sh.smem, st>>>(
        Ab, sA, lda, n, sh.np, sh.lds, sh.vsm, reinterpret_cast<float2*>(G), Vw, 12), note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // The products: FP64 for the FP64 eigendecomposition; double-float on the FP32 pipe (~1e-13
    // relative) when eigenvalues are needed to ~1e-12 ||A|| (polish_tol >= 1e-13)
    const bool df = polish_tol >= 1e-13;
    auto mm = [&](const double2* A_, long lda_, long sA_, const double2* B_, double2* C_) {  // C = A B
      return df ? launch_zgemm_df(n, n, n, A_, lda_, sA_, B_, n, nn, C_, n, nn, nb, st)
                : launch_zgemm(n, n, n, A_, lda_, sA_, B_, n, nn, C_, n, nn, nb, st);
    };
    auto mh = [&](const double2* A_, const double2* B_, double2* C_) {  // C = A^H B
      return df ? launch_zgemm_df_b2(n, n, n, A_, n, nn, 0, B_, n, nn, 0, C_, n, nn, 0, nb, 1, 1, 0, st)
                : launch_zgemm_ah(n, n, n, A_, n, nn, B_, n, nn, C_, n, nn, nb, 0, st);
    };
    // Newton-Schulz: V = Q (I + E) with |E| = d becomes Q (I - 1.5 E^2 + ...): the FP32
    // eigenvectors of an n ~ 100 matrix after a dozen sweeps are unitary only to d ~ 1e-5, so
    // two steps (d^2 ~ 1e-10, then rounding) in either form
    for (int it = 0; it < 2; ++it) {
      if ((e = mh(Vw, Vw, G)) != cudaSuccess) return e;
      if ((e = mm(Vw, n, nn, G, T)) != cudaSuccess) return e;
      const long tot = (long)nb * nn;
      k_ns_update<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(Vw, T, tot), note_launch();
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // A' = V^H (A V)
    if ((e = mm(Ab, lda, sA, Vw, T)) != cudaSuccess) return e;
    if ((e = mh(Vw, T, M)) != cudaSuccess) return e;
    // FP64 sweeps to the first-order finish: angles^2 <= 1e-16 for the FP64 eigendecomposition,
    // 1e-10 (tried right after A') when the eigenvectors are needed to 1e-12
    const double th2 = polish_tol >= 1e-13 ? 1e-10 : 1e-16;
    k_jacobi_polish_big<<<(unsigned)nb, threads_for(nn / 8), 0, st>>>(M, Vw, n, lam, polish_tol, th2,
                                                                       polish_tol >= 1e-13 ? 1 : 0, max_sweeps,
                                                                       status), note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = mm(Vw, n, nn, M, T)) != cudaSuccess) return e;
    k_eig_sort_big<<<(unsigned)nb, threads_for(nn / 4), 0, st>>>(Vw, T, lam, n, w + b0 * sw, sw, V + b0 * sV, sV), note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace eph
