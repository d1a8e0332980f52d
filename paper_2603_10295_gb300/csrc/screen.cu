// Energy-window prescreening of the k list (the step before the interpolation proper in the
// paper's transport workflow: states outside a window around the band edge do not contribute,
// so their k points are dropped before any g(k,q) is formed; the single-node silicon benchmark
// of the Benchmarks section screens k and q with a 0.3 eV window at the conduction band
// minimum, and the practical-guidance discussion notes that the window cuts the contributing
// k points of semiconductors).
//   flag[k] = 1 if some band eps[k][n] lies in [e_lo, e_hi];
//   kept k indices in ascending order by an exclusive scan of the flags (deterministic).
#include "eph_kernels.cuh"

namespace eph {

__global__ void k_window_flags(const double* __restrict__ eps, long nk, int nb, double e_lo, double e_hi,
                               int* __restrict__ flag) {
  const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nk) return;
  int in = 0;
  for (int n = 0; n < nb; ++n) {
    const double e = eps[k * nb + n];
    in |= (e >= e_lo && e <= e_hi) ? 1 : 0;
  }
  flag[k] = in;
}

// Block-level exclusive scan of 1024 flags per block; block totals to tot[blockIdx.x].
__global__ void __launch_bounds__(1024) k_scan_blocks(const int* __restrict__ flag, long n, int* __restrict__ pos,
                                                       int* __restrict__ tot) {
  __shared__ int wsum[32];
  const long i = (long)blockIdx.x * 1024 + threadIdx.x;
  const int v = i < n ? flag[i] : 0;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  if (w == 0) {
    int s = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    wsum[lane] = s;  // inclusive scan of the warp sums
  }
  __syncthreads();
  const int excl = x - v + (w > 0 ? wsum[w - 1] : 0);
  if (i < n) pos[i] = excl;
  if (threadIdx.x == 1023) tot[blockIdx.x] = excl + v;
}

// Serial exclusive scan of the block totals (one thread; the number of blocks is small),
// the grand total to *count.
__global__ void k_scan_totals(int* __restrict__ tot, int nblk, int* __restrict__ count) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int s = 0;
  for (int b = 0; b < nblk; ++b) {
    const int t = tot[b];
    tot[b] = s;
    s += t;
  }
  *count = s;
}

__global__ void k_compact(const int* __restrict__ flag, const int* __restrict__ pos, const int* __restrict__ tot,
                          long n, int* __restrict__ idx) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !flag[i]) return;
  idx[pos[i] + tot[i / 1024]] = (int)i;
}

// out[j][0..2] = kpts[idx[j]][0..2]
__global__ void k_gather_points(const double* __restrict__ kpts, const int* __restrict__ idx, int n,
                                double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const long s = idx[j];
  out[3L * j] = kpts[3 * s];
  out[3L * j + 1] = kpts[3 * s + 1];
  out[3L * j + 2] = kpts[3 * s + 2];
}

// Time-reversal reduction of a uniform k grid (the irreducible k list of the paper's transport
// workflow, for Hamiltonians with real H(Re), where H(-k) = conj H(k) and eps(-k) = eps(k)).
// Grid point i = (j1 n2 + j2) n3 + j3 at k = j/n + s; its partner -k lies on the grid at
// j'_a = (-j_a - t_a) mod n_a, t_a = 2 s_a n_a (an integer).  i is kept if i <= partner(i); a kept
// point stands for itself and its partner: weight 2, or 1 if it is its own partner.
__device__ __forceinline__ long ibz_partner(long i, int n1, int n2, int n3, int t1, int t2, int t3) {
  const int j3 = (int)(i % n3);
  const long r = i / n3;
  const int j2 = (int)(r % n2), j1 = (int)(r / n2);
  auto neg = [](int j, int t, int n) {
    int m = (-j - t) % n;
    return m < 0 ? m + n : m;
  };
  return ((long)neg(j1, t1, n1) * n2 + neg(j2, t2, n2)) * n3 + neg(j3, t3, n3);
}

__global__ void k_ibz_flags(int n1, int n2, int n3, int t1, int t2, int t3, int* __restrict__ flag) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long nk = (long)n1 * n2 * n3;
  if (i >= nk) return;
  flag[i] = i <= ibz_partner(i, n1, n2, n3, t1, t2, t3) ? 1 : 0;
}

__global__ void k_ibz_weights(const int* __restrict__ idx, const int* __restrict__ count, int n1, int n2, int n3,
                              int t1, int t2, int t3, double* __restrict__ w) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= *count) return;
  const long i = idx[j];
  w[j] = ibz_partner(i, n1, n2, n3, t1, t2, t3) == i ? 1.0 : 2.0;
}

cudaError_t launch_ibz_select(int n1, int n2, int n3, const int* t, int* flag, int* pos, int* tot, int* idx,
                              int* count, cudaStream_t st) {
  const long nk = (long)n1 * n2 * n3;
  if (nk <= 0) return cudaSuccess;
  const long nblk = (nk + 1023) / 1024;
  k_ibz_flags<<<(unsigned)((nk + 255) / 256), 256, 0, st>>>(n1, n2, n3, t[0], t[1], t[2], flag), note_launch();
  k_scan_blocks<<<(unsigned)nblk, 1024, 0, st>>>(flag, nk, pos, tot), note_launch();
  k_scan_totals<<<1, 32, 0, st>>>(tot, (int)nblk, count), note_launch();
  k_compact<<<(unsigned)((nk + 255) / 256), 256, 0, st>>>(flag, pos, tot, nk, idx), note_launch();
  return cudaGetLastError();
}

cudaError_t launch_ibz_weights(const int* idx, const int* count, int n_max, int n1, int n2, int n3, const int* t,
                               double* w, cudaStream_t st) {
  if (n_max <= 0) return cudaSuccess;
  k_ibz_weights<<<(n_max + 255) / 256, 256, 0, st>>>(idx, count, n1, n2, n3, t[0], t[1], t[2], w), note_launch();
  return cudaGetLastError();
}

cudaError_t launch_window_select(const double* eps, long nk, int nb, double e_lo, double e_hi, int* flag, int* pos,
                                 int* tot, int* idx, int* count, cudaStream_t st) {
  if (nk <= 0) return cudaSuccess;
  const long nblk = (nk + 1023) / 1024;
  if (nblk > 2147483647L) return cudaErrorInvalidValue;
  k_window_flags<<<(unsigned)((nk + 255) / 256), 256, 0, st>>>(eps, nk, nb, e_lo, e_hi, flag), note_launch();
  k_scan_blocks<<<(unsigned)nblk, 1024, 0, st>>>(flag, nk, pos, tot), note_launch();
  k_scan_totals<<<1, 32, 0, st>>>(tot, (int)nblk, count), note_launch();
  k_compact<<<(unsigned)((nk + 255) / 256), 256, 0, st>>>(flag, pos, tot, nk, idx), note_launch();
  return cudaGetLastError();
}

cudaError_t launch_window_flags(const double* eps, long n, int nb, double e_lo, double e_hi, int* flag,
                                cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_window_flags<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(eps, n, nb, e_lo, e_hi, flag), note_launch();
  return cudaGetLastError();
}

cudaError_t launch_gather_points(const double* kpts, const int* idx, int n, double* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_gather_points<<<(n + 255) / 256, 256, 0, st>>>(kpts, idx, n, out), note_launch();
  return cudaGetLastError();
}

}  // namespace eph
