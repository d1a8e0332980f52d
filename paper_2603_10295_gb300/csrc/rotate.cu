// Rotations of Eq. 10 and phonon post-processing (FP64).
//   mode rotation  G2[q][Re][nu][b] = sum_{ka} u_{ka,nu}(q) G1[q][ka][Re][b]
//                  (applied once per q, before the Re sum, with which it commutes)
//   band rotation  g[q][k][nu] = V_{k+q}^H G3[q][k][nu] V_k   (U_{mm',k+q} U*_{nn',k})
//   phonons        omega = sign(l) sqrt|l| * hbar sqrt(eV/(A^2 amu)), u = e / sqrt(M)
#include <algorithm>

#include "eph_kernels.cuh"

namespace eph {

__global__ void k_phonon_post(const double* __restrict__ lam, const double2* __restrict__ e, int nq, int nm,
                              const double* __restrict__ invsqrtm, double unit, double* __restrict__ omega,
                              double2* __restrict__ u) {
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  long tot = (long)nq * nm * nm;
  if (idx >= tot) return;
  int q = (int)(idx / ((long)nm * nm));
  int rem = (int)(idx - (long)q * nm * nm);
  int r = rem / nm, nu = rem - r * nm;
  double2 ev = e[idx];
  double s = invsqrtm[r];
  u[idx] = make_double2(ev.x * s, ev.y * s);
  if (r == 0) {
    double l = lam[(long)q * nm + nu];
    omega[(long)q * nm + nu] = copysign(sqrt(fabs(l)), l) * unit;
  }
}

cudaError_t launch_phonon_post(const double* lam, const double2* e, int nq, int nm, const double* invsqrtm,
                               double unit, double* omega, double2* u, cudaStream_t st) {
  long tot = (long)nq * nm * nm;
  if (tot <= 0) return cudaSuccess;
  k_phonon_post<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(lam, e, nq, nm, invsqrtm, unit, omega, u), note_launch();
  return cudaGetLastError();
}

// One thread per (q, e, b): reads the nm values G1[q][:][e][b] (coalesced over b),
// writes the nm rotated values.  u[q] is staged in shared memory.
template <int NMX>
__global__ void __launch_bounds__(256) k_mode_rotate(const double2* __restrict__ G1, const double2* __restrict__ u,
                                                     int nm, int ne, int nb2, double2* __restrict__ W, long ldw,
                                                     long sW) {
  __shared__ double2 us[NMX * NMX];
  const int q = blockIdx.y;
  for (int t = threadIdx.x; t < nm * nm; t += blockDim.x) us[t] = u[(long)q * nm * nm + t];
  __syncthreads();
  const long per_q = (long)ne * nb2;
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= per_q) return;
  const int e = (int)(idx / nb2);
  const int b = (int)(idx - (long)e * nb2);
  double2 acc[NMX];
#pragma unroll
  for (int v = 0; v < NMX; ++v) acc[v] = make_double2(0.0, 0.0);
  const double2* src = G1 + (long)q * nm * per_q + (long)e * nb2 + b;
  for (int c = 0; c < nm; ++c) {
    const double2 gv = src[(long)c * per_q];
#pragma unroll
    for (int v = 0; v < NMX; ++v) {
      if (v < nm) {
        const double2 uv = us[c * nm + v];
        acc[v].x = fma(uv.x, gv.x, fma(-uv.y, gv.y, acc[v].x));
        acc[v].y = fma(uv.x, gv.y, fma(uv.y, gv.x, acc[v].y));
      }
    }
  }
  double2* dst = W + (long)q * sW + (long)e * ldw + b;
#pragma unroll
  for (int v = 0; v < NMX; ++v)
    if (v < nm) dst[(long)v * nb2] = acc[v];
}

cudaError_t launch_mode_rotate(const double2* G1, const double2* u, int nq, int nm, int ne, int nb2, double2* W,
                               long ldw, long sW, cudaStream_t st) {
  if (nq <= 0) return cudaSuccess;
  if (nm > 16 || nq > 65535) return cudaErrorInvalidValue;
  long per_q = (long)ne * nb2;
  dim3 grid((unsigned)((per_q + 255) / 256), nq);
  k_mode_rotate<16><<<grid, 256, 0, st>>>(G1, u, nm, ne, nb2, W, ldw, sW), note_launch();
  return cudaGetLastError();
}

// One (q,k) pair of the band rotation in shared memory, three-multiplication complex
// products (3 FMA per complex multiply-add instead of 4) in the form that needs one pre-sum of
// the left operand and two of the right one: for x = a + ib, y = c + id,
//   k1 = c (a + b),  k2 = a (d - c),  k3 = b (c + d),   x y = (k1 - k3) + i (k1 + k2),
// summed over the contraction index with two final additions per output.
//   T = G3_nu V_k:        x = G3 (pre-sum Gr + Gi), y = V_k (pre-sums Vi - Vr, Vr + Vi);
//   g = V_{k+q}^H T:      x = T (pre-sum Tr + Ti), y = conj(V_{k+q}) (pre-sums -Vi - Vr, Vr - Vi).
// Per pair 2 Nb^2 Nm (Nb + 1) + 2 Nb^2 (2 + Nm) + ... : 2,560 additions beside the 18,432 FMA at
// the Si shapes (3,200 with the (re + im) sums of both operands).
struct PairSmem {
  double *ukr, *ukd, *uks;   // V_k: Re, Im - Re, Re + Im
  double *uqr, *uqm, *uqp;   // V_{k+q}: Re, -Im - Re, Re - Im
  double2 *G, *T;
  double *Gs, *Ts;
};

__device__ __forceinline__ PairSmem pair_smem(void* base, int nb, int nm) {
  const int nb2 = nb * nb, x = nm * nb2;
  PairSmem p;
  p.G = static_cast<double2*>(base);
  p.T = p.G + x;
  p.Gs = reinterpret_cast<double*>(p.T + x);
  p.Ts = p.Gs + x;
  p.ukr = p.Ts + x;
  p.ukd = p.ukr + nb2;
  p.uks = p.ukd + nb2;
  p.uqr = p.uks + nb2;
  p.uqm = p.uqr + nb2;
  p.uqp = p.uqm + nb2;
  return p;
}

__host__ __device__ constexpr size_t pair_smem_bytes(int nb, int nm) {
  return (size_t)(2 * nm * nb * nb) * (sizeof(double2) + sizeof(double)) + (size_t)6 * nb * nb * sizeof(double);
}

// Stages the pair and forms T = G3 V_k (all threads of the CTA; ends with a barrier).
__device__ __forceinline__ void pair_stage1(const PairSmem& s, const double2* __restrict__ grow,
                                            const double2* __restrict__ ukg, const double2* __restrict__ ukqg,
                                            int nm, int nb) {
  const int nb2 = nb * nb;
  for (int t = threadIdx.x; t < nb2; t += blockDim.x) {
    const double2 a = ukg[t], b = ukqg[t];
    s.ukr[t] = a.x;
    s.ukd[t] = a.y - a.x;
    s.uks[t] = a.x + a.y;
    s.uqr[t] = b.x;
    s.uqm[t] = -b.y - b.x;
    s.uqp[t] = b.x - b.y;
  }
  for (int t = threadIdx.x; t < nm * nb2; t += blockDim.x) {
    const double2 a = grow[t];
    s.G[t] = a;
    s.Gs[t] = a.x + a.y;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nm * nb2; t += blockDim.x) {
    const int nu = t / nb2, rem = t - nu * nb2, a = rem / nb, n = rem - a * nb;
    const int g0 = nu * nb2 + a * nb;
    double k1 = 0.0, k2 = 0.0, k3 = 0.0;
    for (int b = 0; b < nb; ++b) {
      const double2 x = s.G[g0 + b];
      const int v = b * nb + n;
      k1 = fma(s.ukr[v], s.Gs[g0 + b], k1);
      k2 = fma(x.x, s.ukd[v], k2);
      k3 = fma(x.y, s.uks[v], k3);
    }
    const double2 tv = make_double2(k1 - k3, k1 + k2);
    s.T[t] = tv;
    s.Ts[t] = tv.x + tv.y;
  }
  __syncthreads();
}

// g[nu][m][n] = sum_a conj(V_{k+q}[a][m]) T[nu][a][n] for element t = (nu, m, n).
__device__ __forceinline__ double2 pair_g(const PairSmem& s, int t, int nb) {
  const int nb2 = nb * nb;
  const int nu = t / nb2, rem = t - nu * nb2, m = rem / nb, n = rem - m * nb;
  const int t0 = nu * nb2 + n;
  double k1 = 0.0, k2 = 0.0, k3 = 0.0;
  for (int a = 0; a < nb; ++a) {
    const int v = a * nb + m, ti = t0 + a * nb;
    const double2 y = s.T[ti];
    k1 = fma(s.uqr[v], s.Ts[ti], k1);
    k2 = fma(y.x, s.uqm[v], k2);
    k3 = fma(y.y, s.uqp[v], k3);
  }
  return make_double2(k1 - k3, k1 + k2);
}

// One CTA per (q,k) pair: g_nu = V_{k+q}^H G3_nu V_k (2 nb^3 nm CMAC per pair).  keep (may be
// NULL): pairs with keep[q*nk + k] == 0 are screened out and get g = 0 without any arithmetic.
__global__ void __launch_bounds__(128) k_band_rotate(const double2* __restrict__ Y, long ldy,
                                                     const double2* __restrict__ Ukq,
                                                     const double2* __restrict__ Uk, int nk, int nm, int nb,
                                                     double2* __restrict__ g, long sgq,
                                                     const int* __restrict__ keep) {
  extern __shared__ double2 sm[];
  const PairSmem s = pair_smem(sm, nb, nm);
  const int nb2 = nb * nb;
  const long pair = blockIdx.x;  // q*nk + k
  const int k = (int)(pair % nk);
  const long q = pair / nk;
  double2* out = g + q * sgq + (long)k * nm * nb2;
  if (keep && !keep[pair]) {  // uniform over the CTA: no barrier is skipped by part of it
    for (int t = threadIdx.x; t < nm * nb2; t += blockDim.x) out[t] = make_double2(0.0, 0.0);
    return;
  }
  pair_stage1(s, Y + pair * ldy, Uk + (long)k * nb2, Ukq + pair * nb2, nm, nb);
  for (int t = threadIdx.x; t < nm * nb2; t += blockDim.x) out[t] = pair_g(s, t, nb);
}

cudaError_t launch_band_rotate(const double2* Y, long ldy, const double2* Ukq, const double2* Uk, int nq, int nk,
                               int nm, int nb, double2* g, long sgq, cudaStream_t st, const int* keep) {
  long pairs = (long)nq * nk;
  if (pairs <= 0) return cudaSuccess;
  const size_t smem = pair_smem_bytes(nb, nm);
  if (smem > 220 * 1024) return cudaErrorInvalidValue;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_band_rotate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (pairs > 2147483647L) return cudaErrorInvalidConfiguration;
  k_band_rotate<<<(unsigned)pairs, 128, smem, st>>>(Y, ldy, Ukq, Uk, nk, nm, nb, g, sgq, keep), note_launch();
  return cudaGetLastError();
}

// Persistent band rotation over a mixed work list: segments of (q,k) pairs from several
// contexts (materials of different nb, nm; uneven q batches and k tiles), one launch.  CTAs
// walk the concatenated pair index with a grid stride; each pair finds its segment by binary
// search over the segments' first-pair offsets and runs the same per-pair arithmetic as
// k_band_rotate (bit-identical results), with shared memory sized for the largest segment.
// The segment table travels as a kernel parameter (no host-to-device copy, so the launch can be
// captured in a CUDA graph).
__global__ void __launch_bounds__(128) k_band_rotate_multi(const __grid_constant__ BandSegs segs, int nseg, long total) {
  extern __shared__ double2 sm[];
  for (long t = blockIdx.x; t < total; t += gridDim.x) {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {  // last segment with pair0 <= t
      const int mid = (lo + hi + 1) >> 1;
      if (segs.s[mid].pair0 <= t) lo = mid; else hi = mid - 1;
    }
    const BandSeg& sg = segs.s[lo];
    const int nb = sg.nb, nm = sg.nm, nb2 = nb * nb;
    const PairSmem s = pair_smem(sm, nb, nm);
    const long pair = t - sg.pair0;
    const int k = (int)(pair % sg.nk);
    const long q = pair / sg.nk;
    pair_stage1(s, sg.Y + pair * sg.ldy, sg.Uk + (long)k * nb2, sg.Ukq + pair * nb2, nm, nb);
    double2* out = sg.g + q * sg.sgq + (long)k * nm * nb2;
    for (int e = threadIdx.x; e < nm * nb2; e += blockDim.x) out[e] = pair_g(s, e, nb);
    __syncthreads();  // shared memory is reused by the next pair
  }
}

cudaError_t launch_band_rotate_multi(const BandSegs& segs, int nseg, long total, int max_nb, int max_nm, int nsm,
                                     cudaStream_t st) {
  if (total <= 0 || nseg <= 0) return cudaSuccess;
  if (nseg > kMaxBandSegs || segs.s[0].pair0 != 0) return cudaErrorInvalidValue;
  const size_t smem = pair_smem_bytes(max_nb, max_nm);
  if (smem > 220 * 1024) return cudaErrorInvalidValue;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_band_rotate_multi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_band_rotate_multi, 128, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const long grid = std::min<long>(total, (long)nsm * per_sm);
  k_band_rotate_multi<<<(unsigned)grid, 128, smem, st>>>(segs, nseg, total), note_launch();
  return cudaGetLastError();
}

// Fused consumer: the band rotation of one (q,k) pair into shared memory, then the
// pair's contribution to the electron linewidth of each band n,
//   part[n] = pi w_q sum_{m, nu: omega > omega_min} |g_mn nu|^2 / (2 omega_nu)
//             x [ (n_B + f_m) delta(e_n - e'_m + omega_nu) + (n_B + 1 - f_m) delta(e_n - e'_m - omega_nu) ],
// Gaussian delta of width sigma, n_B = 1/(exp(omega/kT) - 1), f_m = 1/(exp((e'_m - mu)/kT) + 1)
// (e_n = eps_k, e'_m = eps_{k+q}).  g itself is never written to global memory.
__global__ void __launch_bounds__(128) k_band_linewidth(const double2* __restrict__ Y, long ldy,
                                                        const double2* __restrict__ Ukq,
                                                        const double2* __restrict__ Uk,
                                                        const double* __restrict__ epsk,
                                                        const double* __restrict__ epskq,
                                                        const double* __restrict__ om, const double* __restrict__ wq,
                                                        int nk, int nm, int nb, double kT, double mu, double sigma,
                                                        double omega_min, double* __restrict__ part) {
  extern __shared__ double2 sm[];
  const PairSmem s = pair_smem(sm, nb, nm);
  const int nb2 = nb * nb;
  double* fm = reinterpret_cast<double*>(reinterpret_cast<char*>(sm) + pair_smem_bytes(nb, nm));  // [nb] at k+q
  double* nbose = fm + nb;  // [nm] Bose factors (0 for excluded modes)
  const long pair = blockIdx.x;
  const int k = (int)(pair % nk);
  const long q = pair / nk;
  for (int t = threadIdx.x; t < nb; t += blockDim.x) fm[t] = 1.0 / (exp((epskq[pair * nb + t] - mu) / kT) + 1.0);
  for (int t = threadIdx.x; t < nm; t += blockDim.x) {
    const double w = om[q * nm + t];
    nbose[t] = (w > omega_min) ? 1.0 / expm1(w / kT) : 0.0;
  }
  pair_stage1(s, Y + pair * ldy, Uk + (long)k * nb2, Ukq + pair * nb2, nm, nb);
  // each thread forms one g_{m n nu} and its term; the terms overwrite G (free after T)
  const double inv = 1.0 / (sigma * sqrt(2.0 * 3.141592653589793238));
  const double c = -0.5 / (sigma * sigma);
  double* term = reinterpret_cast<double*>(s.G);  // [nu][m][n]
  for (int t = threadIdx.x; t < nm * nb2; t += blockDim.x) {
    const int nu = t / nb2, rem = t - nu * nb2, m = rem / nb, n = rem - m * nb;
    const double w = om[q * nm + nu];
    double v = 0.0;
    if (w > omega_min) {
      const double2 gv = pair_g(s, t, nb);
      const double nB = nbose[nu], f = fm[m];
      const double de = epsk[(long)k * nb + n] - epskq[pair * nb + m];
      const double xa = de + w, xe = de - w;
      const double d = (nB + f) * exp(c * xa * xa) + (nB + 1.0 - f) * exp(c * xe * xe);
      v = fma(gv.x, gv.x, gv.y * gv.y) / (2.0 * w) * d;
    }
    term[t] = v;
  }
  __syncthreads();
  for (int n = threadIdx.x; n < nb; n += blockDim.x) {  // fixed-order sum over (nu, m)
    double s = 0.0;
    for (int j = 0; j < nm * nb; ++j) s += term[j * nb + n];
    part[pair * nb + n] = 3.141592653589793238 * wq[q] * inv * s;
  }
}

cudaError_t launch_band_linewidth(const double2* Y, long ldy, const double2* Ukq, const double2* Uk, const double* epsk,
                                  const double* epskq, const double* om, const double* wq, int nq, int nk, int nm,
                                  int nb, double kT, double mu, double sigma, double omega_min, double* part,
                                  cudaStream_t st) {
  const long pairs = (long)nq * nk;
  if (pairs <= 0) return cudaSuccess;
  const size_t smem = pair_smem_bytes(nb, nm) + (size_t)(nb + nm) * sizeof(double);
  if (smem > 220 * 1024) return cudaErrorInvalidValue;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_band_linewidth, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (pairs > 2147483647L) return cudaErrorInvalidConfiguration;
  k_band_linewidth<<<(unsigned)pairs, 128, smem, st>>>(Y, ldy, Ukq, Uk, epsk, epskq, om, wq, nk, nm, nb, kT, mu, sigma,
                                                       omega_min, part), note_launch();
  return cudaGetLastError();
}

// The same linewidth terms from g rows already formed ([nu][m][n] of a pair at G + pair ldg): one
// CTA per pair; thread t takes column n = n0 + t % cols and every rpp-th row (nu, m) from t / cols,
// its partial sums then combine in a fixed order (deterministic for any nb, nm).
__global__ void __launch_bounds__(128) k_linewidth_terms(const double2* __restrict__ G, long ldg,
                                                         const double* __restrict__ epsk,
                                                         const double* __restrict__ epskq,
                                                         const double* __restrict__ om, const double* __restrict__ wq,
                                                         int nk, int nm, int nb, double kT, double mu, double sigma,
                                                         double omega_min, double* __restrict__ part) {
  extern __shared__ double lw_sm[];
  double* fm = lw_sm;         // [nb] Fermi factors at k+q
  double* nbose = fm + nb;    // [nm] Bose factors (0 for excluded modes)
  double* red = nbose + nm;   // [blockDim.x] partial sums
  const long pair = blockIdx.x;
  const int k = (int)(pair % nk);
  const long q = pair / nk;
  for (int t = threadIdx.x; t < nb; t += blockDim.x) fm[t] = 1.0 / (exp((epskq[pair * nb + t] - mu) / kT) + 1.0);
  for (int t = threadIdx.x; t < nm; t += blockDim.x) {
    const double w = om[q * nm + t];
    nbose[t] = (w > omega_min) ? 1.0 / expm1(w / kT) : 0.0;
  }
  __syncthreads();
  const double inv = 1.0 / (sigma * sqrt(2.0 * 3.141592653589793238));
  const double c = -0.5 / (sigma * sigma);
  const double2* g = G + pair * ldg;
  const int R = nm * nb;  // rows (nu, m)
  for (int n0 = 0; n0 < nb; n0 += blockDim.x) {
    const int cols = min(nb - n0, (int)blockDim.x);
    const int rpp = blockDim.x / cols;
    const int n = n0 + threadIdx.x % cols, r1 = threadIdx.x / cols;
    double sum = 0.0;
    if (r1 < rpp) {
      const double en = epsk[(long)k * nb + n];
      for (int r = r1; r < R; r += rpp) {
        const int nu = r / nb, m = r - nu * nb;
        const double w = om[q * nm + nu];
        if (w > omega_min) {
          const double2 gv = g[(long)r * nb + n];
          const double nB = nbose[nu], f = fm[m];
          const double de = en - epskq[pair * nb + m];
          const double xa = de + w, xe = de - w;
          const double d = (nB + f) * exp(c * xa * xa) + (nB + 1.0 - f) * exp(c * xe * xe);
          sum += fma(gv.x, gv.x, gv.y * gv.y) / (2.0 * w) * d;
        }
      }
    }
    red[threadIdx.x] = sum;
    __syncthreads();
    if ((int)threadIdx.x < cols) {
      double tot = 0.0;
      for (int i = 0; i < rpp; ++i) tot += red[i * cols + threadIdx.x];
      part[pair * nb + n] = 3.141592653589793238 * wq[q] * inv * tot;
    }
    __syncthreads();
  }
}

cudaError_t launch_linewidth_terms(const double2* G, long ldg, const double* epsk, const double* epskq,
                                   const double* om, const double* wq, int nq, int nk, int nm, int nb, double kT,
                                   double mu, double sigma, double omega_min, double* part, cudaStream_t st) {
  const long pairs = (long)nq * nk;
  if (pairs <= 0) return cudaSuccess;
  if (pairs > 2147483647L) return cudaErrorInvalidConfiguration;
  const size_t smem = (size_t)(nb + nm + 128) * sizeof(double);
  k_linewidth_terms<<<(unsigned)pairs, 128, smem, st>>>(G, ldg, epsk, epskq, om, wq, nk, nm, nb, kT, mu, sigma,
                                                        omega_min, part), note_launch();
  return cudaGetLastError();
}

// acc[k][n] += sum_{q < nq} part[q][k][n] (fixed order over q).
__global__ void k_sum_over_q(const double* __restrict__ part, int nq, long per_q, double* __restrict__ acc) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= per_q) return;
  double s = acc[idx];
  for (int q = 0; q < nq; ++q) s += part[(long)q * per_q + idx];
  acc[idx] = s;
}

cudaError_t launch_sum_over_q(const double* part, int nq, long per_q, double* acc, cudaStream_t st) {
  if (per_q <= 0 || nq <= 0) return cudaSuccess;
  k_sum_over_q<<<(unsigned)((per_q + 255) / 256), 256, 0, st>>>(part, nq, per_q, acc), note_launch();
  return cudaGetLastError();
}

}  // namespace eph
