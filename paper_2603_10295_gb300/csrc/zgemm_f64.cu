// FP64 complex contractions on the DFMA pipe.
//
// On GB300 the FP64 pipe issues about two DFMA per clock per SM, so these
// kernels are bound by FP64 arithmetic, not by memory: a 64x64 register tile
// per 256-thread CTA with 8-deep shared-memory staging keeps the pipe fed, and
// the tiled GEMM spends three DFMA per complex multiply-add (3M form).
//   - k_zgemm:   C = A B or C (+)= A^H B   (Fourier sums over Re: H(k), H(k+q),
//                Re->k of g (Eq. 10); adjoint sums over k and q)
//   - k_skinny:  few rows times a wide operand (Rp->q of g, Eq. 9; D(q))
#include "eph_kernels.cuh"

namespace eph {

namespace {
constexpr int BM = 64, BN = 64, BK = 8;

__device__ __forceinline__ void cmac(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
}  // namespace

// ADJ: op(A) = A^H with A stored K x M (row stride lda).  ACC: C += result.
// Complex products use the 3-multiplication form (Gauss / "3M"): with the pre-added
// sums s_a = a_r + a_i and s_b = b_r + b_i staged once per shared-memory tile,
//   t1 += a_r b_r,  t2 += a_i b_i,  t3 += s_a s_b,   C = (t1 - t2) + i (t3 - t1 - t2),
// i.e. three DFMA per complex multiply-add instead of four.
// Batch index z = b1 * nbat2 + b2 with operand offsets b1 s*1 + b2 s*2 (nbat2 = 1: plain batch).
template <bool ADJ, bool ACC>
__global__ void __launch_bounds__(256) k_zgemm(int M, int N, int K, const double2* __restrict__ A, long lda,
                                               long sA, const double2* __restrict__ B, long ldb, long sB,
                                               double2* __restrict__ C, long ldc, long sC, int nbat2, long sA2,
                                               long sB2, long sC2) {
  __shared__ double3 As[BK][BM];  // (re, im, re + im)
  __shared__ double3 Bs[BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  // grid.x runs over (column block, batch) with the column block fastest, so the CTAs
  // that share one row block of A (all batches) run back to back and reuse it from L2
  const int nN = (N + BN - 1) / BN;
  const long z = blockIdx.x / nN;
  const int m0 = blockIdx.y * BM, n0 = (int)(blockIdx.x - z * nN) * BN;
  const long b1 = z / nbat2, b2 = z - b1 * nbat2;
  A += b1 * sA + b2 * sA2;
  B += b1 * sB + b2 * sB2;
  C += b1 * sC + b2 * sC2;
  double t1[4][4], t2[4][4], t3[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) t1[i][j] = t2[i][j] = t3[i][j] = 0.0;

  for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      int idx = tid + 256 * l;
      double2 v;
      int am, ak;
      if (!ADJ) {
        am = idx >> 3;
        ak = idx & 7;
        const int gm = m0 + am, gk = k0 + ak;
        v = (gm < M && gk < K) ? A[(long)gm * lda + gk] : make_double2(0.0, 0.0);
      } else {
        ak = idx >> 6;
        am = idx & 63;
        const int gm = m0 + am, gk = k0 + ak;
        v = (gm < M && gk < K) ? A[(long)gk * lda + gm] : make_double2(0.0, 0.0);
        v.y = -v.y;
      }
      As[ak][am] = make_double3(v.x, v.y, v.x + v.y);
      {
        int kk = idx >> 6, n = idx & 63;
        int gn = n0 + n, gk = k0 + kk;
        const double2 w = (gn < N && gk < K) ? B[(long)gk * ldb + gn] : make_double2(0.0, 0.0);
        Bs[kk][n] = make_double3(w.x, w.y, w.x + w.y);
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double3 a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          t1[i][j] = fma(a[i].x, bb[j].x, t1[i][j]);
          t2[i][j] = fma(a[i].y, bb[j].y, t2[i][j]);
          t3[i][j] = fma(a[i].z, bb[j].z, t3[i][j]);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      const double2 r = make_double2(t1[i][j] - t2[i][j], t3[i][j] - t1[i][j] - t2[i][j]);
      double2* p = C + (long)gm * ldc + gn;
      if (ACC) {
        double2 o = *p;
        *p = make_double2(o.x + r.x, o.y + r.y);
      } else {
        *p = r;
      }
    }
  }
}

static bool grid_ok(int M, int N, int batch) {
  return M > 0 && N > 0 && batch > 0 && (M + BM - 1) / BM <= 65535 && batch <= 65535;
}

cudaError_t launch_zgemm(int M, int N, int K, const double2* A, long lda, long sA, const double2* B, long ldb,
                         long sB, double2* C, long ldc, long sC, int batch, cudaStream_t st) {
  if (M <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
  if (!grid_ok(M, N, batch)) return cudaErrorInvalidConfiguration;
  dim3 grid((unsigned)(((N + BN - 1) / BN) * batch), (M + BM - 1) / BM, 1);
  k_zgemm<false, false><<<grid, 256, 0, st>>>(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC, 1, 0, 0, 0), note_launch();
  return cudaGetLastError();
}

cudaError_t launch_zgemm_b2(int M, int N, int K, const double2* A, long lda, long sA, long sA2, const double2* B,
                            long ldb, long sB, long sB2, double2* C, long ldc, long sC, long sC2, int nbat1,
                            int nbat2, int adj, cudaStream_t st) {
  const long batch = (long)nbat1 * nbat2;
  if (M <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
  if (batch > 65535 || !grid_ok(M, N, 1)) return cudaErrorInvalidConfiguration;
  dim3 grid((unsigned)(((N + BN - 1) / BN) * batch), (M + BM - 1) / BM, 1);
  if (adj)
    k_zgemm<true, false><<<grid, 256, 0, st>>>(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC, nbat2, sA2, sB2, sC2), note_launch();
  else
    k_zgemm<false, false><<<grid, 256, 0, st>>>(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC, nbat2, sA2, sB2, sC2), note_launch();
  return cudaGetLastError();
}

cudaError_t launch_zgemm_ah(int M, int N, int K, const double2* A, long lda, long sA, const double2* B, long ldb,
                            long sB, double2* C, long ldc, long sC, int batch, int acc, cudaStream_t st) {
  if (M <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
  if (!grid_ok(M, N, batch)) return cudaErrorInvalidConfiguration;
  dim3 grid((unsigned)(((N + BN - 1) / BN) * batch), (M + BM - 1) / BM, 1);
  if (acc)
    k_zgemm<true, true><<<grid, 256, 0, st>>>(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC, 1, 0, 0, 0), note_launch();
  else
    k_zgemm<true, false><<<grid, 256, 0, st>>>(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC, 1, 0, 0, 0), note_launch();
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Skinny: C[m][x] = sum_r P[m][r] B[r][x] for M <= MQ rows (a q batch).
// One thread per column x; the M x 64 phase chunk sits in shared memory and is
// broadcast, B is streamed once with coalesced loads.
// ----------------------------------------------------------------------------
template <int MQ, bool REAL_B>
__global__ void __launch_bounds__(256) k_skinny(int M, long N, int K, const double2* __restrict__ P, long ldp,
                                                const void* __restrict__ Bv, long ldb,
                                                const double* __restrict__ colscale, double2* __restrict__ C,
                                                long ldc) {
  constexpr int RC = 64;
  __shared__ double2 Ps[MQ][RC];
  const long x = (long)blockIdx.x * blockDim.x + threadIdx.x;
  double2 acc[MQ];
#pragma unroll
  for (int m = 0; m < MQ; ++m) acc[m] = make_double2(0.0, 0.0);
  for (int r0 = 0; r0 < K; r0 += RC) {
    for (int t = threadIdx.x; t < MQ * RC; t += blockDim.x) {
      int m = t / RC, rr = t - m * RC;
      Ps[m][rr] = (m < M && r0 + rr < K) ? P[(long)m * ldp + r0 + rr] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    if (x < N) {
      int rn = min(RC, K - r0);
      for (int rr = 0; rr < rn; ++rr) {
        if (REAL_B) {
          double bv = static_cast<const double*>(Bv)[(long)(r0 + rr) * ldb + x];
#pragma unroll
          for (int m = 0; m < MQ; ++m) {
            acc[m].x = fma(Ps[m][rr].x, bv, acc[m].x);
            acc[m].y = fma(Ps[m][rr].y, bv, acc[m].y);
          }
        } else {
          double2 bv = static_cast<const double2*>(Bv)[(long)(r0 + rr) * ldb + x];
#pragma unroll
          for (int m = 0; m < MQ; ++m) cmac(acc[m], Ps[m][rr], bv);
        }
      }
    }
    __syncthreads();
  }
  if (x < N) {
    double s = colscale ? colscale[x] : 1.0;
#pragma unroll
    for (int m = 0; m < MQ; ++m)
      if (m < M) C[(long)m * ldc + x] = make_double2(acc[m].x * s, acc[m].y * s);
  }
}

template <bool REAL_B>
static cudaError_t skinny_dispatch(int M, long N, int K, const double2* P, long ldp, const void* B, long ldb,
                                   const double* cs, double2* C, long ldc, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (M > 16) return cudaErrorInvalidValue;
  int threads = 256;
  unsigned blocks = (unsigned)((N + threads - 1) / threads);
#define EPH_SK(MQ)                                                                                   \
  case MQ:                                                                                           \
    k_skinny<MQ, REAL_B><<<blocks, threads, 0, st>>>(M, N, K, P, ldp, B, ldb, cs, C, ldc), note_launch(); \
    break;
  switch (M) {
    EPH_SK(1) EPH_SK(2) EPH_SK(3) EPH_SK(4) EPH_SK(5) EPH_SK(6) EPH_SK(7) EPH_SK(8)
    EPH_SK(9) EPH_SK(10) EPH_SK(11) EPH_SK(12) EPH_SK(13) EPH_SK(14) EPH_SK(15) EPH_SK(16)
    default: return cudaErrorInvalidValue;
  }
#undef EPH_SK
  return cudaGetLastError();
}

cudaError_t launch_skinny(int M, long N, int K, const double2* P, long ldp, const double2* B, long ldb, double2* C,
                          long ldc, cudaStream_t st) {
  return skinny_dispatch<false>(M, N, K, P, ldp, B, ldb, nullptr, C, ldc, st);
}

cudaError_t launch_skinny_real(int M, long N, int K, const double2* P, long ldp, const double* B, long ldb,
                               const double* colscale, double2* C, long ldc, cudaStream_t st) {
  return skinny_dispatch<true>(M, N, K, P, ldp, B, ldb, colscale, C, ldc, st);
}

// Plain transpose of a batch of square matrices: out[b][j][i] = in[b][i][j].
__global__ void k_transpose(const double2* __restrict__ in, int n, long batch, double2* __restrict__ out) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long nn = (long)n * n;
  if (idx >= nn * batch) return;
  const long b = idx / nn;
  const int r = (int)((idx - b * nn) / n), c = (int)(idx - b * nn - (long)r * n);
  out[b * nn + (long)c * n + r] = in[idx];
}

cudaError_t launch_transpose(const double2* in, int n, long batch, double2* out, cudaStream_t st) {
  const long tot = (long)n * n * batch;
  if (tot <= 0) return cudaSuccess;
  k_transpose<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(in, n, batch, out), note_launch();
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Double-float complex GEMM on the FP32 pipe: C = A B with FP64 inputs and output,
// every operand carried as a pair of floats (hi + lo, ~48 bits) and every product
// formed exactly with an FMA and accumulated with a two-sum.  Relative error
// ~1e-13 of the sum of |terms|, at about one fifth of the DFMA time on GB300
// (12 FP32 operations per real multiply-add at 64x the FP64 rate).  Used where
// FP64-class accuracy is needed but not FP64 itself (H(k+q) for the mixed form).
// ----------------------------------------------------------------------------
namespace {
struct ff2 {  // complex double-float: (re_hi, re_lo, im_hi, im_lo)
  float rh, rl, ih, il;
};
__device__ __forceinline__ float4 to_ff(double2 v) {
  const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
  return make_float4(rh, __double2float_rn(v.x - (double)rh), ih, __double2float_rn(v.y - (double)ih));
}
// (sh, sl) += (ah + al)(bh + bl); products error-free via FMA, sum via two-sum.
// __fmul_rn/__fadd_rn are never contracted into FMAs, which the transforms rely on.
__device__ __forceinline__ void dfmac(float& sh, float& sl, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  const float s = __fadd_rn(sh, p);
  const float bb = __fsub_rn(s, sh);
  sl = __fadd_rn(sl, __fadd_rn(__fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(p, bb)), e));
  sh = s;
}
}  // namespace

// C = op(A) B in double-float arithmetic on the FP32 pipe (~1e-14 relative); op(A) = A or
// A^H (ADJ); C complex128 or complex64 (OUT32); batch index z = b1 * nbat2 + b2 with operand
// offsets b1 s*1 + b2 s*2.
template <bool ADJ, bool OUT32>
__global__ void __launch_bounds__(256, 2) k_zgemm_df(int M, int N, int K, const double2* __restrict__ A, long lda,
                                                  long sA, const double2* __restrict__ B, long ldb, long sB,
                                                  void* __restrict__ Cv, long ldc, long sC, int nbat2, long sA2,
                                                  long sB2, long sC2) {
  __shared__ float4 As[BK][BM];
  __shared__ float4 Bs[BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int nN = (N + BN - 1) / BN;  // grid.x = (column block, batch), column block fastest
  const long z = blockIdx.x / nN;
  const int m0 = blockIdx.y * BM, n0 = (int)(blockIdx.x - z * nN) * BN;
  const long b1 = z / nbat2, b2 = z - b1 * nbat2;
  A += b1 * sA + b2 * sA2;
  B += b1 * sB + b2 * sB2;
  const long coff = b1 * sC + b2 * sC2;
  ff2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = ff2{0.f, 0.f, 0.f, 0.f};
  for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      const int idx = tid + 256 * l;
      {
        const int m = idx >> 3, kk = idx & 7, gm = m0 + m, gk = k0 + kk;
        double2 av = make_double2(0.0, 0.0);
        if (gm < M && gk < K) {
          if (ADJ) {
            av = A[(long)gk * lda + gm];
            av.y = -av.y;
          } else {
            av = A[(long)gm * lda + gk];
          }
        }
        As[kk][m] = to_ff(av);
      }
      {
        const int kk = idx >> 6, n = idx & 63, gn = n0 + n, gk = k0 + kk;
        Bs[kk][n] = to_ff((gn < N && gk < K) ? B[(long)gk * ldb + gn] : make_double2(0.0, 0.0));
      }
    }
    __syncthreads();
#pragma unroll 2
    for (int kk = 0; kk < BK; ++kk) {
      float4 a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          ff2& c = acc[i][j];
          // (ar + i ai)(br + i bi): re += ar br - ai bi, im += ar bi + ai br
          dfmac(c.rh, c.rl, a[i].x, a[i].y, bb[j].x, bb[j].y);
          dfmac(c.rh, c.rl, -a[i].z, -a[i].w, bb[j].z, bb[j].w);
          dfmac(c.ih, c.il, a[i].x, a[i].y, bb[j].z, bb[j].w);
          dfmac(c.ih, c.il, a[i].z, a[i].w, bb[j].x, bb[j].y);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      const ff2& c = acc[i][j];
      if (OUT32)
        static_cast<float2*>(Cv)[coff + (long)gm * ldc + gn] = make_float2(__fadd_rn(c.rh, c.rl), __fadd_rn(c.ih, c.il));
      else
        static_cast<double2*>(Cv)[coff + (long)gm * ldc + gn] =
            make_double2((double)c.rh + (double)c.rl, (double)c.ih + (double)c.il);
    }
  }
}

cudaError_t launch_zgemm_df(int M, int N, int K, const double2* A, long lda, long sA, const double2* B, long ldb,
                            long sB, double2* C, long ldc, long sC, int batch, cudaStream_t st) {
  if (M <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
  if (!grid_ok(M, N, batch)) return cudaErrorInvalidConfiguration;
  dim3 grid((unsigned)(((N + BN - 1) / BN) * batch), (M + BM - 1) / BM, 1);
  k_zgemm_df<false, false><<<grid, 256, 0, st>>>(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC, 1, 0, 0, 0), note_launch();
  return cudaGetLastError();
}

cudaError_t launch_zgemm_df_b2(int M, int N, int K, const double2* A, long lda, long sA, long sA2, const double2* B,
                               long ldb, long sB, long sB2, void* C, long ldc, long sC, long sC2, int nbat1, int nbat2,
                               int adj, int out32, cudaStream_t st) {
  const long batch = (long)nbat1 * nbat2;
  if (M <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
  if (batch > 65535 || !grid_ok(M, N, 1)) return cudaErrorInvalidConfiguration;
  dim3 grid((unsigned)(((N + BN - 1) / BN) * batch), (M + BM - 1) / BM, 1);
#define EPH_DF(ADJV, O32)                                                                                         \
  k_zgemm_df<ADJV, O32><<<grid, 256, 0, st>>>(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC, nbat2, sA2, sB2, sC2), note_launch()
  if (adj && out32)
    EPH_DF(true, true);
  else if (adj)
    EPH_DF(true, false);
  else if (out32)
    EPH_DF(false, true);
  else
    EPH_DF(false, false);
#undef EPH_DF
  return cudaGetLastError();
}

}  // namespace eph
