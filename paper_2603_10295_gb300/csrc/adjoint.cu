// Hand-written adjoint of the interpolation (Eqs. 9-10) for the scalar
//   L = sum_{q,k,nu,m,n} c_{q k nu n} |g_mnnu(k,q)|^2,  c = w_nk / omega_qnu (omega > omega_min, else 0)
// with the eigenvectors V_k, V_{k+q} and u(q) held fixed.  With g = A(gW) linear,
// dL/dRe(gW) + i dL/dIm(gW) = A^H(2 c g), applied in reverse order:
//   gbar = 2 c g;  G3bar_nu = V_{k+q} gbar_nu V_k^H;  G2bar = sum_k conj(P_k) G3bar;
//   G1bar[ka] = sum_nu conj(u_{ka,nu}) G2bar[nu];  grad = sum_q conj(P_q(Rp)) G1bar.
// The Re->k contraction G3 is recomputed per k tile, never stored across tiles.
#include "eph_kernels.cuh"

namespace eph {

// G3bar[nu] = V_{k+q} gbar[nu] V_k^H for one pair, all threads of the CTA:
// gbar in G (shared), T shared scratch of nm nb^2, result to the row (global).
__device__ __forceinline__ void back_rotate(const double2* G, double2* T, const double2* uk, const double2* ukq,
                                            int nm, int nb, double2* row) {
  const int nb2 = nb * nb;
  // S[nu][m][b] = sum_n gbar[nu][m][n] conj(uk[b][n])   (in T)
  for (int t = threadIdx.x; t < nm * nb2; t += blockDim.x) {
    const int nu = t / nb2, rem = t - nu * nb2, m = rem / nb, b = rem - m * nb;
    double2 acc = make_double2(0.0, 0.0);
    for (int n = 0; n < nb; ++n) {
      const double2 x = G[nu * nb2 + m * nb + n], y = uk[b * nb + n];
      acc.x = fma(x.x, y.x, fma(x.y, y.y, acc.x));
      acc.y = fma(x.y, y.x, fma(-x.x, y.y, acc.y));
    }
    T[t] = acc;
  }
  __syncthreads();
  // G3bar[nu][a][b] = sum_m ukq[a][m] S[nu][m][b]  -> back into the row
  for (int t = threadIdx.x; t < nm * nb2; t += blockDim.x) {
    const int nu = t / nb2, rem = t - nu * nb2, a = rem / nb, b = rem - a * nb;
    double2 acc = make_double2(0.0, 0.0);
    for (int m = 0; m < nb; ++m) {
      const double2 x = ukq[a * nb + m], y = T[nu * nb2 + m * nb + b];
      acc.x = fma(x.x, y.x, fma(-x.y, y.y, acc.x));
      acc.y = fma(x.x, y.y, fma(x.y, y.x, acc.y));
    }
    row[t] = acc;
  }
}

// Per (q,k) pair: g from G3 (band rotation), L_pair = sum c |g|^2, then
// G3bar = V_{k+q} (2 c g) V_k^H written over the pair's G3 row in place.
__global__ void __launch_bounds__(128) k_band_adjoint(double2* __restrict__ Y, long ldy,
                                                      const double2* __restrict__ Ukq, const double2* __restrict__ Uk,
                                                      const double* __restrict__ wk, const double* __restrict__ om,
                                                      double omega_min, int nk, int nm, int nb,
                                                      double* __restrict__ Lpair) {
  extern __shared__ double2 sm[];
  __shared__ double red[4];
  const int nb2 = nb * nb;
  double2* uk = sm;
  double2* ukq = uk + nb2;
  double2* G = ukq + nb2;
  double2* T = G + nm * nb2;
  const long pair = blockIdx.x;
  const int k = (int)(pair % nk);
  const int q = (int)(pair / nk);
  double2* row = Y + pair * ldy;
  for (int t = threadIdx.x; t < nb2; t += blockDim.x) {
    uk[t] = Uk[(long)k * nb2 + t];
    ukq[t] = Ukq[pair * nb2 + t];
  }
  for (int t = threadIdx.x; t < nm * nb2; t += blockDim.x) G[t] = row[t];
  __syncthreads();
  // T[nu][a][n] = sum_b G[nu][a][b] uk[b][n]
  for (int t = threadIdx.x; t < nm * nb2; t += blockDim.x) {
    const int nu = t / nb2, rem = t - nu * nb2, a = rem / nb, n = rem - a * nb;
    double2 acc = make_double2(0.0, 0.0);
    for (int b = 0; b < nb; ++b) {
      const double2 x = G[nu * nb2 + a * nb + b], y = uk[b * nb + n];
      acc.x = fma(x.x, y.x, fma(-x.y, y.y, acc.x));
      acc.y = fma(x.x, y.y, fma(x.y, y.x, acc.y));
    }
    T[t] = acc;
  }
  __syncthreads();
  // g[nu][m][n] = sum_a conj(ukq[a][m]) T[nu][a][n]; gbar = 2 c g (stored in G); L partial
  double lsum = 0.0;
  for (int t = threadIdx.x; t < nm * nb2; t += blockDim.x) {
    const int nu = t / nb2, rem = t - nu * nb2, m = rem / nb, n = rem - m * nb;
    double2 acc = make_double2(0.0, 0.0);
    for (int a = 0; a < nb; ++a) {
      const double2 x = ukq[a * nb + m], y = T[nu * nb2 + a * nb + n];
      acc.x = fma(x.x, y.x, fma(x.y, y.y, acc.x));
      acc.y = fma(x.x, y.y, fma(-x.y, y.x, acc.y));
    }
    const double w = om[(long)q * nm + nu];
    const double c = (w > omega_min) ? wk[(long)k * nb + n] / w : 0.0;
    lsum = fma(c, fma(acc.x, acc.x, acc.y * acc.y), lsum);
    G[t] = make_double2(2.0 * c * acc.x, 2.0 * c * acc.y);
  }
  __syncthreads();
  back_rotate(G, T, uk, ukq, nm, nb, row);
  // deterministic block reduction of the pair's L
  for (int off = 16; off > 0; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lsum;
  __syncthreads();
  if (threadIdx.x == 0) Lpair[pair] = red[0] + red[1] + red[2] + red[3];
}

cudaError_t launch_band_adjoint(double2* Y, long ldy, const double2* Ukq, const double2* Uk, const double* wk,
                                const double* om, double omega_min, int nq, int nk, int nm, int nb, double* Lpair,
                                cudaStream_t st) {
  long pairs = (long)nq * nk;
  if (pairs <= 0) return cudaSuccess;
  size_t smem = (size_t)(2 * nb * nb + 2 * nm * nb * nb) * sizeof(double2);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_band_adjoint, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (pairs > 2147483647L) return cudaErrorInvalidConfiguration;
  k_band_adjoint<<<(unsigned)pairs, 128, smem, st>>>(Y, ldy, Ukq, Uk, wk, om, omega_min, nk, nm, nb, Lpair), note_launch();
  return cudaGetLastError();
}

// Vector-Jacobian product of the band rotation for an arbitrary upstream gradient:
// G3bar = V_{k+q} gbar V_k^H written over the pair's G3 row (gbar[q][k][nu][m][n] with
// q stride sgq).
__global__ void __launch_bounds__(128) k_band_vjp(double2* __restrict__ Y, long ldy, const double2* __restrict__ gbar,
                                                  long sgq, const double2* __restrict__ Ukq,
                                                  const double2* __restrict__ Uk, int nk, int nm, int nb) {
  extern __shared__ double2 sm[];
  const int nb2 = nb * nb;
  double2* uk = sm;
  double2* ukq = uk + nb2;
  double2* G = ukq + nb2;
  double2* T = G + nm * nb2;
  const long pair = blockIdx.x;
  const int k = (int)(pair % nk);
  const long q = pair / nk;
  const double2* gb = gbar + q * sgq + (long)k * nm * nb2;
  for (int t = threadIdx.x; t < nb2; t += blockDim.x) {
    uk[t] = Uk[(long)k * nb2 + t];
    ukq[t] = Ukq[pair * nb2 + t];
  }
  for (int t = threadIdx.x; t < nm * nb2; t += blockDim.x) G[t] = gb[t];
  __syncthreads();
  back_rotate(G, T, uk, ukq, nm, nb, Y + pair * ldy);
}

cudaError_t launch_band_vjp(double2* Y, long ldy, const double2* gbar, long sgq, const double2* Ukq,
                            const double2* Uk, int nq, int nk, int nm, int nb, cudaStream_t st) {
  const long pairs = (long)nq * nk;
  if (pairs <= 0) return cudaSuccess;
  const size_t smem = (size_t)(2 * nb * nb + 2 * nm * nb * nb) * sizeof(double2);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_band_vjp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (pairs > 2147483647L) return cudaErrorInvalidConfiguration;
  k_band_vjp<<<(unsigned)pairs, 128, smem, st>>>(Y, ldy, gbar, sgq, Ukq, Uk, nk, nm, nb), note_launch();
  return cudaGetLastError();
}

// Loss terms of the adjoint for large shapes, one CTA per (q,k) pair over the pair's g row
// [nu][m][n] (row stride ldy): Lpair = sum c |g|^2 in a fixed order, and 2 c g written in place,
// c = w_nk / omega_qnu (0 for omega <= omega_min).
__global__ void __launch_bounds__(256) k_loss_terms(double2* __restrict__ Y, long ldy, const double* __restrict__ wk,
                                                    const double* __restrict__ om, double omega_min, int nk, int nm,
                                                    int nb, double* __restrict__ Lpair) {
  __shared__ double red[8];
  const long pair = blockIdx.x;
  const int k = (int)(pair % nk);
  const long q = pair / nk;
  const int nb2 = nb * nb;
  double2* row = Y + pair * ldy;
  double lsum = 0.0;
  for (int nu = 0; nu < nm; ++nu) {
    const double w = om[q * nm + nu];
    const double inv = w > omega_min ? 1.0 / w : 0.0;
    for (int t = threadIdx.x; t < nb2; t += blockDim.x) {
      const int n = t % nb;
      const double c = wk[(long)k * nb + n] * inv;
      const double2 g = row[(long)nu * nb2 + t];
      lsum = fma(c, fma(g.x, g.x, g.y * g.y), lsum);
      row[(long)nu * nb2 + t] = make_double2(2.0 * c * g.x, 2.0 * c * g.y);
    }
  }
  for (int off = 16; off > 0; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < 8; ++i) t += red[i];
    Lpair[pair] = t;
  }
}

cudaError_t launch_loss_terms(double2* Y, long ldy, const double* wk, const double* om, double omega_min, int nq,
                              int nk, int nm, int nb, double* Lpair, cudaStream_t st) {
  const long pairs = (long)nq * nk;
  if (pairs <= 0) return cudaSuccess;
  if (pairs > 2147483647L) return cudaErrorInvalidConfiguration;
  k_loss_terms<<<(unsigned)pairs, 256, 0, st>>>(Y, ldy, wk, om, omega_min, nk, nm, nb, Lpair), note_launch();
  return cudaGetLastError();
}

// g = 0 on the pairs (q, k) with keep[q nk + k] == 0: pair (q, k) holds `per` elements of `eb` bytes
// at g + (q sgq + k per) eb (a block of threads per pair; eb = 8 or 16)
__global__ void k_zero_masked(char* __restrict__ g, int eb, long sgq, long per, int nk, const int* __restrict__ keep) {
  const long pair = blockIdx.x;
  if (keep[pair]) return;
  const long q = pair / nk, k = pair - q * nk;
  char* base = g + (q * sgq + k * per) * eb;
  const long words = per * eb / 8;
  for (long i = threadIdx.x; i < words; i += blockDim.x) reinterpret_cast<unsigned long long*>(base)[i] = 0ULL;
}

cudaError_t launch_zero_masked(void* g, int eb, long sgq, long per, int nq, int nk, const int* keep, cudaStream_t st) {
  const long pairs = (long)nq * nk;
  if (pairs <= 0 || !keep) return cudaSuccess;
  if ((eb != 8 && eb != 16) || pairs > 2147483647L || (reinterpret_cast<uintptr_t>(g) & 7)) return cudaErrorInvalidValue;
  k_zero_masked<<<(unsigned)pairs, 128, 0, st>>>(static_cast<char*>(g), eb, sgq, per, nk, keep), note_launch();
  return cudaGetLastError();
}

// out[b][j][i] = conj(in[b][i][j]) for a batch of n x n complex matrices (V^H of eigenvector sets)
__global__ void k_conj_transpose(const double2* __restrict__ in, int n, long total, double2* __restrict__ out) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  const long nn = (long)n * n, b = t / nn;
  const int r = (int)(t - b * nn), i = r / n, j = r - i * n;
  const double2 v = in[t];
  out[b * nn + (long)j * n + i] = make_double2(v.x, -v.y);
}

cudaError_t launch_conj_transpose(const double2* in, int n, long batch, double2* out, cudaStream_t st) {
  const long total = batch * n * n;
  if (total <= 0) return cudaSuccess;
  k_conj_transpose<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(in, n, total, out), note_launch();
  return cudaGetLastError();
}

// f[c] = s M_c with M_c = 1 / invsqrtm[c]^2 (the mass of mode index c = 3 kappa + alpha).
__global__ void k_mass_factors(const double* __restrict__ invsqrtm, int nm, double s, double* __restrict__ f) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < nm) f[c] = s / (invsqrtm[c] * invsqrtm[c]);
}

cudaError_t launch_mass_factors(const double* invsqrtm, int nm, double s, double* f, cudaStream_t st) {
  if (nm <= 0) return cudaSuccess;
  k_mass_factors<<<(nm + 127) / 128, 128, 0, st>>>(invsqrtm, nm, s, f), note_launch();
  return cudaGetLastError();
}

// X[q][c][i] *= f[c] for i < blk (in place).
__global__ void k_scale_modes(double2* __restrict__ X, long per_q, long blk, const double* __restrict__ f, long n) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const long c = (idx % per_q) / blk;
  const double s = f[c];
  const double2 v = X[idx];
  X[idx] = make_double2(v.x * s, v.y * s);
}

cudaError_t launch_scale_modes(double2* X, int nq, int nm, long blk, const double* f, cudaStream_t st) {
  const long n = (long)nq * nm * blk;
  if (n <= 0) return cudaSuccess;
  k_scale_modes<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(X, (long)nm * blk, blk, f, n), note_launch();
  return cudaGetLastError();
}

// Sum of n partial values into *L (one CTA, fixed order: deterministic).
__global__ void __launch_bounds__(256) k_sum_into(const double* __restrict__ v, long n, double* __restrict__ L) {
  __shared__ double red[8];
  double s = 0.0;
  for (long i = threadIdx.x; i < n; i += blockDim.x) s += v[i];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < 8; ++i) t += red[i];
    *L += t;
  }
}

cudaError_t launch_sum_into(const double* v, long n, double* L, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_sum_into<<<1, 256, 0, st>>>(v, n, L), note_launch();
  return cudaGetLastError();
}

// G1bar[q][c][e][b] = sum_nu conj(u[q][c][nu]) G2bar[q][e][nu][b]
template <int NMX>
__global__ void __launch_bounds__(256) k_mode_rotate_adj(const double2* __restrict__ G2b, const double2* __restrict__ u,
                                                         int nm, int ne, int nb2, double2* __restrict__ G1b) {
  __shared__ double2 us[NMX * NMX];
  const int q = blockIdx.y;
  for (int t = threadIdx.x; t < nm * nm; t += blockDim.x) us[t] = u[(long)q * nm * nm + t];
  __syncthreads();
  const long per_q = (long)ne * nb2;
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= per_q) return;
  const int e = (int)(idx / nb2);
  const int b = (int)(idx - (long)e * nb2);
  double2 val[NMX];
  const double2* src = G2b + (long)q * nm * per_q + (long)e * nm * nb2 + b;
#pragma unroll
  for (int v = 0; v < NMX; ++v) val[v] = (v < nm) ? src[(long)v * nb2] : make_double2(0.0, 0.0);
  double2* dst = G1b + (long)q * nm * per_q + (long)e * nb2 + b;
  for (int c = 0; c < nm; ++c) {
    double2 acc = make_double2(0.0, 0.0);
#pragma unroll
    for (int v = 0; v < NMX; ++v) {
      if (v < nm) {
        const double2 x = us[c * nm + v], y = val[v];
        acc.x = fma(x.x, y.x, fma(x.y, y.y, acc.x));
        acc.y = fma(x.x, y.y, fma(-x.y, y.x, acc.y));
      }
    }
    dst[(long)c * per_q] = acc;
  }
}

cudaError_t launch_mode_rotate_adj(const double2* G2b, const double2* u, int nq, int nm, int ne, int nb2, double2* G1b,
                                   cudaStream_t st) {
  if (nq <= 0) return cudaSuccess;
  if (nm > 16 || nq > 65535) return cudaErrorInvalidValue;
  long per_q = (long)ne * nb2;
  dim3 grid((unsigned)((per_q + 255) / 256), nq);
  k_mode_rotate_adj<16><<<grid, 256, 0, st>>>(G2b, u, nm, ne, nb2, G1b), note_launch();
  return cudaGetLastError();
}

}  // namespace eph
