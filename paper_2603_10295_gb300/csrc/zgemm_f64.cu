// FP64 complex contractions on the DFMA pipe.
//
// On GB300 the FP64 pipe issues about two DFMA per clock per SM, so these
// kernels are bound by FP64 arithmetic, not by memory: a 64x64 register tile
// per 256-thread CTA with 8-deep shared-memory staging keeps the pipe fed.
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
template <bool ADJ, bool ACC>
__global__ void __launch_bounds__(256) k_zgemm(int M, int N, int K, const double2* __restrict__ A, long lda,
                                               long sA, const double2* __restrict__ B, long ldb, long sB,
                                               double2* __restrict__ C, long ldc, long sC) {
  __shared__ double2 As[BK][BM];
  __shared__ double2 Bs[BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const long b = blockIdx.z;
  A += b * sA;
  B += b * sB;
  C += b * sC;
  double2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_double2(0.0, 0.0);

  for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      int idx = tid + 256 * l;
      if (!ADJ) {
        int m = idx >> 3, kk = idx & 7;
        int gm = m0 + m, gk = k0 + kk;
        As[kk][m] = (gm < M && gk < K) ? A[(long)gm * lda + gk] : make_double2(0.0, 0.0);
      } else {
        int kk = idx >> 6, m = idx & 63;
        int gm = m0 + m, gk = k0 + kk;
        double2 v = (gm < M && gk < K) ? A[(long)gk * lda + gm] : make_double2(0.0, 0.0);
        As[kk][m] = make_double2(v.x, -v.y);
      }
      {
        int kk = idx >> 6, n = idx & 63;
        int gn = n0 + n, gk = k0 + kk;
        Bs[kk][n] = (gn < N && gk < K) ? B[(long)gk * ldb + gn] : make_double2(0.0, 0.0);
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double2 a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) cmac(acc[i][j], a[i], bb[j]);
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
      double2* p = C + (long)gm * ldc + gn;
      if (ACC) {
        double2 o = *p;
        *p = make_double2(o.x + acc[i][j].x, o.y + acc[i][j].y);
      } else {
        *p = acc[i][j];
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
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, batch);
  k_zgemm<false, false><<<grid, 256, 0, st>>>(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC);
  return cudaGetLastError();
}

cudaError_t launch_zgemm_ah(int M, int N, int K, const double2* A, long lda, long sA, const double2* B, long ldb,
                            long sB, double2* C, long ldc, long sC, int batch, int acc, cudaStream_t st) {
  if (M <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
  if (!grid_ok(M, N, batch)) return cudaErrorInvalidConfiguration;
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, batch);
  if (acc)
    k_zgemm<true, true><<<grid, 256, 0, st>>>(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC);
  else
    k_zgemm<true, false><<<grid, 256, 0, st>>>(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC);
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
    k_skinny<MQ, REAL_B><<<blocks, threads, 0, st>>>(M, N, K, P, ldp, B, ldb, cs, C, ldc); \
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

}  // namespace eph
