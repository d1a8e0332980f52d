// Phase factors of the interpolation formula (paper Eq. 7; split per stage in Eqs. 9-10):
// P[i][r] = w_r exp(2 pi i k_i . R_r), k in crystal coordinates, R integer.
// The argument t = k.n is formed in FP64 and reduced exactly, r = t - rint(t)
// (Sterbenz: the subtraction is exact), before sincospi(2r).
#include "eph_kernels.cuh"

namespace eph {

__global__ void k_phase(const double* __restrict__ pts, int n, const int* __restrict__ R,
                        const double* __restrict__ w, int nR, double2* __restrict__ P, long ldp) {
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  long total = (long)n * nR;
  if (idx >= total) return;
  int i = (int)(idx / nR);
  int r = (int)(idx - (long)i * nR);
  const double k0 = pts[3 * i], k1 = pts[3 * i + 1], k2 = pts[3 * i + 2];
  const double n0 = (double)R[3 * r], n1 = (double)R[3 * r + 1], n2 = (double)R[3 * r + 2];
  double t = fma(k2, n2, fma(k1, n1, k0 * n0));
  double red = t - rint(t);
  double s, c;
  sincospi(2.0 * red, &s, &c);
  double wr = w ? w[r] : 1.0;
  P[(long)i * ldp + r] = make_double2(wr * c, wr * s);
}

cudaError_t launch_phase(const double* pts, int n, const int* R, const double* w, int nR, double2* P,
                         long ldp, cudaStream_t st) {
  long total = (long)n * nR;
  if (total <= 0) return cudaSuccess;
  int threads = 256;
  long blocks = (total + threads - 1) / threads;
  k_phase<<<(unsigned)blocks, threads, 0, st>>>(pts, n, R, w, nR, P, ldp), note_launch();
  return cudaGetLastError();
}

// B[q][e][j] = Q[q][e] * H[e][j]: the per-q right operand of the H(k+q) transform,
// sum_e w_e e^{i k.e} (e^{i q.e} H(e)) = H(k+q).
__global__ void k_scale_rows(const double2* __restrict__ Q, int nq, const double2* __restrict__ H, int ne,
                             int cols, double2* __restrict__ B, long ldb, long sB) {
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  long per_q = (long)ne * cols;
  if (idx >= per_q * nq) return;
  int q = (int)(idx / per_q);
  long rem = idx - (long)q * per_q;
  int e = (int)(rem / cols);
  int j = (int)(rem - (long)e * cols);
  B[(long)q * sB + (long)e * ldb + j] = cmul(Q[(long)q * ne + e], H[(long)e * cols + j]);
}

cudaError_t launch_scale_rows(const double2* Q, int nq, const double2* H, int ne, int cols, double2* B,
                              long ldb, long sB, cudaStream_t st) {
  long total = (long)nq * ne * cols;
  if (total <= 0) return cudaSuccess;
  int threads = 256;
  k_scale_rows<<<(unsigned)((total + threads - 1) / threads), threads, 0, st>>>(Q, nq, H, ne, cols, B, ldb,
                                                                                sB), note_launch();
  return cudaGetLastError();
}

}  // namespace eph
