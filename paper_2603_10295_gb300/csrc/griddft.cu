// Re->k contraction on a product k grid (Eq. 10, and the H(k+q) sum of Eq. 4), by sum
// factorisation.  On k = (j1/N1 + s1, j2/N2 + s2, j3/N3 + s3) the phase of a lattice vector
// n = (n1, n2, n3) factorises, e^{2 pi i k.n} = prod_a e^{2 pi i (j_a/N_a + s_a) n_a}, so with
// the Re list scattered into a box of slots b = (b1, b2, b3) (zeros where no Re vector lies),
//   Y[j1 j2 j3][c] = sum_b1 E1[j1][b1] sum_b2 E2[j2][b2] sum_b3 E3[j3][b3] Wbox[b1 b2 b3][c]
// is three small DFTs along one axis each (B_a terms per output instead of |Re|).  Every
// product of the definition appears once: the result equals the direct sum up to rounding.
// Slots are symmetric: along an axis of half-width M, slot 0 holds n = 0 and slots 2m - 1,
// 2m hold n = +m, -m (m = 1..M), so that a whole unshifted axis pairs e^{i t m} with
// e^{-i t m} (see k_axis_dft).
#include "eph_kernels.cuh"

namespace eph {

__host__ __device__ __forceinline__ int slot_n(int b) { return b == 0 ? 0 : ((b & 1) ? (b + 1) / 2 : -(b / 2)); }

// E[j][b] = exp(2 pi i (j/N + s) n(b)).  The argument is reduced exactly: j n mod N in
// integers, then frac(s n) formed in FP64 and reduced like the k.R argument of k_phase.
__global__ void k_axis_phase(int N, int B, double shift, double2* __restrict__ E) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N * B) return;
  const int j = idx / B, b = idx - j * B;
  const long n = slot_n(b);
  long m = ((long)j * n) % N;
  if (m < 0) m += N;
  double t = (double)m / (double)N;
  const double sn = shift * (double)n;
  t += sn - rint(sn);
  const double r = t - rint(t);
  double s, c;
  sincospi(2.0 * r, &s, &c);
  E[idx] = make_double2(c, s);
}

cudaError_t launch_axis_phase(int N, int B, double shift, double2* E, cudaStream_t st) {
  const int total = N * B;
  if (total <= 0) return cudaSuccess;
  k_axis_phase<<<(total + 255) / 256, 256, 0, st>>>(N, B, shift, E), note_launch();
  return cudaGetLastError();
}

// Wbox[q][box[e]][c] = w_e W[q][e][c] (Wbox zeroed beforehand; box[] is injective).
__global__ void k_box_scatter(const double2* __restrict__ W, long sWq, long ldw, int ne, int ncols,
                              const int* __restrict__ box, const double* __restrict__ we, double2* __restrict__ Wbox,
                              long sBq, int nq) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long per_q = (long)ne * ncols;
  if (idx >= per_q * nq) return;
  const int q = (int)(idx / per_q);
  const long rem = idx - (long)q * per_q;
  const int e = (int)(rem / ncols);
  const int c = (int)(rem - (long)e * ncols);
  const double2 v = W[q * sWq + (long)e * ldw + c];
  const double w = we[e];
  Wbox[q * sBq + (long)box[e] * ncols + c] = make_double2(w * v.x, w * v.y);
}

cudaError_t launch_box_scatter(const double2* W, long sWq, long ldw, int ne, int ncols, const int* box,
                               const double* we, double2* Wbox, long sBq, int nq, cudaStream_t st) {
  const long total = (long)nq * ne * ncols;
  if (total <= 0) return cudaSuccess;
  k_box_scatter<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(W, sWq, ldw, ne, ncols, box, we, Wbox, sBq, nq), note_launch();
  return cudaGetLastError();
}

// One axis: out[a][j - j0][c] = sum_{b < B} E[j][b] in[a][b][c] for j0 <= j < j0 + nj.
// One thread per (a, c): the B inputs stay in registers, E (nj x B) is broadcast from shared
// memory.  paired: the range is the whole axis with no shift (B = 2M + 1 symmetric slots), so
// with u_m = x_{+m} + x_{-m}, w_m = x_{+m} - x_{-m} and (c, s) = E[j][2m - 1],
//   A = x_0 + sum_m c u_m,  B = sum_m s w_m,  out[j] = A + i B,  out[N - j] = A - i B:
// 2M + 2 FP64 operations per output instead of 3B (the three-multiplication form used for
// shifted axes and partial ranges).
// BMAX = B exactly (odd: symmetric slots), so no predicated-off FP64 instruction is issued.
template <int BMAX>
__global__ void __launch_bounds__(256) k_axis_dft(const double2* __restrict__ in, long sa_in, long C, int B,
                                                  const double2* __restrict__ E, int N, int j0, int nj, int paired,
                                                  double2* __restrict__ out, long sa_out) {
  extern __shared__ double2 es[];  // [nj][B]
  const int a = blockIdx.y;
  for (int t = threadIdx.x; t < nj * BMAX; t += blockDim.x) es[t] = E[(long)j0 * BMAX + t];
  __syncthreads();
  const long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  double xr[BMAX], xi[BMAX];
  const double2* src = in + (long)a * sa_in + c;
#pragma unroll
  for (int b = 0; b < BMAX; ++b) {
    const double2 v = src[(long)b * C];
    xr[b] = v.x;
    xi[b] = v.y;
  }
  double2* dst = out + (long)a * sa_out + c;
  if (paired) {
    constexpr int MM = (BMAX - 1) / 2;  // BMAX odd: slots 2m - 1, 2m < BMAX for m <= MM
    double ur[MM + 1], ui[MM + 1], wr[MM + 1], wi[MM + 1];
#pragma unroll
    for (int m = 1; m <= MM; ++m) {
      ur[m - 1] = xr[2 * m - 1] + xr[2 * m];
      ui[m - 1] = xi[2 * m - 1] + xi[2 * m];
      wr[m - 1] = xr[2 * m - 1] - xr[2 * m];
      wi[m - 1] = xi[2 * m - 1] - xi[2 * m];
    }
    for (int j = 0; 2 * j <= N; ++j) {
      const double2* e = es + j * BMAX;
      double ar = xr[0], ai = xi[0], br = 0.0, bi = 0.0;
#pragma unroll
      for (int m = 1; m <= MM; ++m) {
        const double2 w = e[2 * m - 1];
        ar = fma(w.x, ur[m - 1], ar);
        ai = fma(w.x, ui[m - 1], ai);
        br = fma(w.y, wr[m - 1], br);
        bi = fma(w.y, wi[m - 1], bi);
      }
      dst[(long)j * C] = make_double2(ar - bi, ai + br);
      const int jm = N - j;
      if (j != 0 && jm != j) dst[(long)jm * C] = make_double2(ar + bi, ai - br);
    }
  } else {
    double xs[BMAX];
#pragma unroll
    for (int b = 0; b < BMAX; ++b) xs[b] = xr[b] + xi[b];
    for (int j = 0; j < nj; ++j) {
      const double2* e = es + j * BMAX;
      double t1 = 0.0, t2 = 0.0, t3 = 0.0;  // sum er xr, ei xi, (er + ei)(xr + xi)
#pragma unroll
      for (int b = 0; b < BMAX; ++b) {
        const double2 w = e[b];
        t1 = fma(w.x, xr[b], t1);
        t2 = fma(w.y, xi[b], t2);
        t3 = fma(w.x + w.y, xs[b], t3);
      }
      dst[(long)j * C] = make_double2(t1 - t2, t3 - t1 - t2);
    }
  }
}

// The paired transform in double-float arithmetic on the FP32 pipe (GB300's FP64 unit runs at
// ~1/64 of its FP32 rate): every FP64 value is split into a float pair (hi, lo), hi the nearest
// float and lo the nearest float to the remainder (48 significant bits, relative 2^-48), products
// are formed exactly with an FMA (two-product) and accumulated with error-free two-sums, and each
// output is joined back to a double.  The splits and joins take the integer-operation conversions
// below plus one FP64 addition per real value: ~2 FP64 operations per output instead of ~8.
// Accuracy ~2^-46 of the largest term of each output (the FP64 kernel: ~2^-53).
namespace {
__device__ __forceinline__ float d2f_rn_i(double x) {  // nearest float (normal range), integer operations
  const unsigned long long b = (unsigned long long)__double_as_longlong(x) + (1ULL << 28);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned e = (hi >> 20) & 0x7FFu;
  const unsigned mag = __funnelshift_l(lo, hi, 3) - (896u << 23);
  return (e > 896u && e < 1151u) ? __uint_as_float(mag | (hi & 0x80000000u)) : 0.f;
}
__device__ __forceinline__ double f2d_exact_i(float x) {  // exact, integer operations
  const unsigned u = __float_as_uint(x);
  const unsigned e = (u >> 23) & 0xFFu;
  if (e == 0u) return 0.0;
  const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7FFFFFu) >> 3);
  return __hiloint2double((int)hi, (int)(u << 29));
}
struct DF {
  float h, l;
};
__device__ __forceinline__ DF df_split(double x) {
  const float h = d2f_rn_i(x);
  return DF{h, d2f_rn_i(x - f2d_exact_i(h))};
}
__device__ __forceinline__ double df_join(float s, float t) { return f2d_exact_i(s) + f2d_exact_i(t); }
// (S, T) += a b: the product's rounding error from an FMA, the sum's from a two-sum
__device__ __forceinline__ void df_fma(float& S, float& T, DF a, DF b) {
  const float p = __fmul_rn(a.h, b.h);
  const float pe = __fmaf_rn(a.h, b.h, -p);
  const float t = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, pe));
  const float s = __fadd_rn(S, p);
  const float bb = __fsub_rn(s, S);
  const float e = __fadd_rn(__fsub_rn(S, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  S = s;
  T = __fadd_rn(T, __fadd_rn(e, t));
}
// (S1, T1) + sg (S2, T2) rounded to FP32 (sg = +-1): the head sum by a two-sum, no FP64 operation
__device__ __forceinline__ float df_addf(float S1, float T1, float S2, float T2, float sg) {
  const float b2 = sg * S2;
  const float s = __fadd_rn(S1, b2);
  const float bb = __fsub_rn(s, S1);
  const float e = __fadd_rn(__fsub_rn(S1, __fsub_rn(s, bb)), __fsub_rn(b2, bb));
  return __fadd_rn(s, __fadd_rn(__fadd_rn(T1, sg * T2), e));
}
// (S1, T1) + sg (S2, T2) joined to a double (sg = +-1)
__device__ __forceinline__ double df_addj(float S1, float T1, float S2, float T2, float sg) {
  const float b2 = sg * S2;
  const float s = __fadd_rn(S1, b2);
  const float bb = __fsub_rn(s, S1);
  const float e = __fadd_rn(__fsub_rn(S1, __fsub_rn(s, bb)), __fsub_rn(b2, bb));
  return df_join(s, __fadd_rn(__fadd_rn(T1, sg * T2), e));
}
}  // namespace

// With out32, column c of every row of nw columns whose index c mod nw is >= nd is written as
// complex64 to out32[a][j][c / nw][c mod nw - nd] (rows of nw - nd) instead of to out: the
// consumer of those columns needs FP32 only, and they skip the FP64 joins.
template <int BMAX>
__global__ void __launch_bounds__(256) k_axis_dft_df(const double2* __restrict__ in, long sa_in, long C,
                                                     const double2* __restrict__ E, int N,
                                                     double2* __restrict__ out, long sa_out, int nw, int nd,
                                                     float2* __restrict__ out32, long sa_out32) {
  constexpr int MM = (BMAX - 1) / 2;
  extern __shared__ float4 ef[];  // [N / 2 + 1][MM]: (cos hi, cos lo, sin hi, sin lo) of slot 2m - 1
  const int a = blockIdx.y;
  const int nh = N / 2 + 1;
  for (int t = threadIdx.x; t < nh * MM; t += blockDim.x) {
    const int j = t / MM, m = t - j * MM + 1;
    const double2 w = E[(long)j * BMAX + 2 * m - 1];
    const DF c = df_split(w.x), sn = df_split(w.y);
    ef[t] = make_float4(c.h, c.l, sn.h, sn.l);
  }
  __syncthreads();
  const long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  const double2* src = in + (long)a * sa_in + c;
  DF x0r, x0i, ur[MM > 0 ? MM : 1], ui[MM > 0 ? MM : 1], wr[MM > 0 ? MM : 1], wi[MM > 0 ? MM : 1];
  {
    const double2 v0 = src[0];
    x0r = df_split(v0.x);
    x0i = df_split(v0.y);
#pragma unroll
    for (int m = 1; m <= MM; ++m) {
      const double2 p = src[(long)(2 * m - 1) * C], q = src[(long)(2 * m) * C];
      ur[m - 1] = df_split(p.x + q.x);
      ui[m - 1] = df_split(p.y + q.y);
      wr[m - 1] = df_split(p.x - q.x);
      wi[m - 1] = df_split(p.y - q.y);
    }
  }
  double2* dst = out + (long)a * sa_out + c;
  const int cw = out32 ? (int)(c % nw) : 0;
  const bool f32o = out32 != nullptr && cw >= nd;
  const long C32 = out32 ? (C / nw) * (nw - nd) : 0;
  float2* dst32 = f32o ? out32 + (long)a * sa_out32 + (c / nw) * (nw - nd) + (cw - nd) : nullptr;
  for (int j = 0; 2 * j <= N; ++j) {
    float arS = x0r.h, arT = x0r.l, aiS = x0i.h, aiT = x0i.l, brS = 0.f, brT = 0.f, biS = 0.f, biT = 0.f;
#pragma unroll
    for (int m = 0; m < MM; ++m) {
      const float4 w = ef[j * MM + m];
      const DF cm{w.x, w.y}, sm{w.z, w.w};
      df_fma(arS, arT, cm, ur[m]);
      df_fma(aiS, aiT, cm, ui[m]);
      df_fma(brS, brT, sm, wr[m]);
      df_fma(biS, biT, sm, wi[m]);
    }
    const int jm = N - j;
    if (f32o) {
      dst32[(long)j * C32] = make_float2(df_addf(arS, arT, biS, biT, -1.f), df_addf(aiS, aiT, brS, brT, 1.f));
      if (j != 0 && jm != j)
        dst32[(long)jm * C32] = make_float2(df_addf(arS, arT, biS, biT, 1.f), df_addf(aiS, aiT, brS, brT, -1.f));
    } else {
      dst[(long)j * C] = make_double2(df_addj(arS, arT, biS, biT, -1.f), df_addj(aiS, aiT, brS, brT, 1.f));
      if (j != 0 && jm != j)
        dst[(long)jm * C] = make_double2(df_addj(arS, arT, biS, biT, 1.f), df_addj(aiS, aiT, brS, brT, -1.f));
    }
  }
}

cudaError_t launch_axis_dft_df(const double2* in, long sa_in, int A, long C, int B, const double2* E, int N,
                               double2* out, long sa_out, cudaStream_t st, int nw, int nd, float2* out32,
                               long sa_out32) {
  if (A <= 0 || C <= 0) return cudaSuccess;
  if (B < 1 || B > 33 || (B & 1) == 0 || A > 65535) return cudaErrorInvalidValue;
  if (out32 && (nw < 1 || nd < 0 || nd > nw || C % nw != 0)) return cudaErrorInvalidValue;
  const size_t smem = (size_t)(N / 2 + 1) * ((B - 1) / 2 > 0 ? (B - 1) / 2 : 1) * sizeof(float4);
  if (smem > 48 * 1024) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)((C + 255) / 256), (unsigned)A, 1);
  auto go = [&](auto kern) -> cudaError_t {
    kern<<<grid, 256, smem, st>>>(in, sa_in, C, E, N, out, sa_out, nw, nd, out32, sa_out32), note_launch();
    return cudaGetLastError();
  };
  switch (B) {
#define EPH_AXIS_B(V) \
  case V:             \
    return go(k_axis_dft_df<V>);
    EPH_AXIS_B(1) EPH_AXIS_B(3) EPH_AXIS_B(5) EPH_AXIS_B(7) EPH_AXIS_B(9) EPH_AXIS_B(11) EPH_AXIS_B(13)
    EPH_AXIS_B(15) EPH_AXIS_B(17) EPH_AXIS_B(19) EPH_AXIS_B(21) EPH_AXIS_B(23) EPH_AXIS_B(25) EPH_AXIS_B(27)
    EPH_AXIS_B(29) EPH_AXIS_B(31) EPH_AXIS_B(33)
#undef EPH_AXIS_B
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_axis_dft(const double2* in, long sa_in, int A, long C, int B, const double2* E, int N, int j0,
                            int nj, int paired, double2* out, long sa_out, cudaStream_t st) {
  if (A <= 0 || C <= 0 || nj <= 0) return cudaSuccess;
  if (B < 1 || B > 33 || (B & 1) == 0 || A > 65535 || j0 < 0 || j0 + nj > N) return cudaErrorInvalidValue;
  if (paired && (j0 != 0 || nj != N)) return cudaErrorInvalidValue;
  const size_t smem = (size_t)nj * B * sizeof(double2);
  if (smem > 160 * 1024) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)((C + 255) / 256), (unsigned)A, 1);
  auto go = [&](auto kern) -> cudaError_t {
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    kern<<<grid, 256, smem, st>>>(in, sa_in, C, B, E, N, j0, nj, paired, out, sa_out), note_launch();
    return cudaGetLastError();
  };
  switch (B) {
#define EPH_AXIS_B(V) \
  case V:             \
    return go(k_axis_dft<V>);
    EPH_AXIS_B(1) EPH_AXIS_B(3) EPH_AXIS_B(5) EPH_AXIS_B(7) EPH_AXIS_B(9) EPH_AXIS_B(11) EPH_AXIS_B(13)
    EPH_AXIS_B(15) EPH_AXIS_B(17) EPH_AXIS_B(19) EPH_AXIS_B(21) EPH_AXIS_B(23) EPH_AXIS_B(25) EPH_AXIS_B(27)
    EPH_AXIS_B(29) EPH_AXIS_B(31) EPH_AXIS_B(33)
#undef EPH_AXIS_B
    default:
      return cudaErrorInvalidValue;  // the slot box has odd extents only
  }
}

// Adjoint of one axis transform (the Re <- k direction of the backward pass, Eq. 10 transposed):
//   out[a][b][r][c] (+)= sum_{j0 <= j < j0 + nj} conj(E[j][b]) in[a][j - j0][r][c]
// for every slot b < B, row r < R and column c < CC.  One thread per (a, r, c) keeps the B
// complex accumulators in registers and streams the nj inputs once; conj(E) comes from shared
// memory.  Four DFMA per (j, b) and output column.
template <int BMAX>
__global__ void __launch_bounds__(256) k_axis_adj(const double2* __restrict__ in, long sa_in, long sj_in, long ldr_in,
                                                  int R, int CC, const double2* __restrict__ E, int j0, int nj,
                                                  double2* __restrict__ out, long sa_out, long sb_out, long ldr_out,
                                                  int accumulate) {
  extern __shared__ double2 es[];  // [nj][BMAX]
  const int a = blockIdx.y;
  for (int t = threadIdx.x; t < nj * BMAX; t += blockDim.x) es[t] = E[(long)j0 * BMAX + t];
  __syncthreads();
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)R * CC) return;
  const int r = (int)(idx / CC), c = (int)(idx - (long)r * CC);
  double ar[BMAX], ai[BMAX];
  double2* dst = out + (long)a * sa_out + (long)r * ldr_out + c;
#pragma unroll
  for (int b = 0; b < BMAX; ++b) {
    if (accumulate) {
      const double2 v = dst[(long)b * sb_out];
      ar[b] = v.x;
      ai[b] = v.y;
    } else {
      ar[b] = 0.0;
      ai[b] = 0.0;
    }
  }
  const double2* src = in + (long)a * sa_in + (long)r * ldr_in + c;
  for (int j = 0; j < nj; ++j) {
    const double2 x = src[(long)j * sj_in];
    const double2* e = es + j * BMAX;
#pragma unroll
    for (int b = 0; b < BMAX; ++b) {  // conj(e) x
      const double2 w = e[b];
      ar[b] = fma(w.x, x.x, ar[b]);
      ar[b] = fma(w.y, x.y, ar[b]);
      ai[b] = fma(w.x, x.y, ai[b]);
      ai[b] = fma(-w.y, x.x, ai[b]);
    }
  }
#pragma unroll
  for (int b = 0; b < BMAX; ++b) dst[(long)b * sb_out] = make_double2(ar[b], ai[b]);
}

// The same adjoint over a whole unshifted axis (j0 = 0, nj = N, symmetric slots): E[N - j] =
// conj(E[j]) and slot 2m holds conj of slot 2m - 1, so with S = x_j + x_{N-j}, D = x_{N-j} - x_j
// (S = x_j, D = -x_j when j has no partner) and (c, s) = E[j][2m - 1],
//   out[2m - 1] += c S + i s D,  out[2m] += c S - i s D,  out[0] += S:
// two real products per complex term for two slots and two j, a quarter of the FP64 operations.
template <int BMAX>
__global__ void __launch_bounds__(256) k_axis_adj_paired(const double2* __restrict__ in, long sa_in, long sj_in,
                                                         long ldr_in, int R, int CC, const double2* __restrict__ E,
                                                         int N, double2* __restrict__ out, long sa_out, long sb_out,
                                                         long ldr_out, int accumulate) {
  constexpr int MM = (BMAX - 1) / 2;
  extern __shared__ double2 eo[];  // [N / 2 + 1][MM]: E[j][2m - 1]
  const int a = blockIdx.y;
  const int nh = N / 2 + 1;
  for (int t = threadIdx.x; t < nh * MM; t += blockDim.x) {
    const int j = t / MM, m = t - j * MM + 1;
    eo[t] = E[(long)j * BMAX + 2 * m - 1];
  }
  __syncthreads();
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)R * CC) return;
  const int r = (int)(idx / CC), c = (int)(idx - (long)r * CC);
  double pr[MM > 0 ? MM : 1], pi[MM > 0 ? MM : 1], qr[MM > 0 ? MM : 1], qi[MM > 0 ? MM : 1];
#pragma unroll
  for (int m = 0; m < MM; ++m) pr[m] = pi[m] = qr[m] = qi[m] = 0.0;
  double s0r = 0.0, s0i = 0.0;
  const double2* src = in + (long)a * sa_in + (long)r * ldr_in + c;
  for (int j = 0; 2 * j <= N; ++j) {
    const int jm = N - j;
    const double2 x = src[(long)j * sj_in];
    double Sr = x.x, Si = x.y, Dr = -x.x, Di = -x.y;
    if (j != 0 && jm != j) {
      const double2 y = src[(long)jm * sj_in];
      Sr = x.x + y.x;
      Si = x.y + y.y;
      Dr = y.x - x.x;
      Di = y.y - x.y;
    }
    s0r += Sr;
    s0i += Si;
    const double2* e = eo + j * MM;
#pragma unroll
    for (int m = 0; m < MM; ++m) {
      const double2 w = e[m];
      pr[m] = fma(w.x, Sr, pr[m]);
      pi[m] = fma(w.x, Si, pi[m]);
      qr[m] = fma(w.y, Dr, qr[m]);
      qi[m] = fma(w.y, Di, qi[m]);
    }
  }
  double2* dst = out + (long)a * sa_out + (long)r * ldr_out + c;
  auto put = [&](int b, double vr, double vi) {
    double2* o = dst + (long)b * sb_out;
    if (accumulate) {
      const double2 v = *o;
      vr += v.x;
      vi += v.y;
    }
    *o = make_double2(vr, vi);
  };
  put(0, s0r, s0i);
#pragma unroll
  for (int m = 0; m < MM; ++m) {
    put(2 * m + 1, pr[m] - qi[m], pi[m] + qr[m]);  // c S + i s D
    put(2 * m + 2, pr[m] + qi[m], pi[m] - qr[m]);  // c S - i s D
  }
}

cudaError_t launch_axis_adj_paired(const double2* in, long sa_in, long sj_in, long ldr_in, int A, int R, int CC, int B,
                                   const double2* E, int N, double2* out, long sa_out, long sb_out, long ldr_out,
                                   int accumulate, cudaStream_t st) {
  if (A <= 0 || R <= 0 || CC <= 0 || N <= 0) return cudaSuccess;
  if (B < 1 || B > 33 || (B & 1) == 0 || A > 65535) return cudaErrorInvalidValue;
  const size_t smem = (size_t)(N / 2 + 1) * (B > 1 ? (B - 1) / 2 : 1) * sizeof(double2);
  if (smem > 48 * 1024) return cudaErrorInvalidValue;
  const long cols = (long)R * CC;
  const dim3 grid((unsigned)((cols + 255) / 256), (unsigned)A, 1);
  auto go = [&](auto kern) -> cudaError_t {
    kern<<<grid, 256, smem, st>>>(in, sa_in, sj_in, ldr_in, R, CC, E, N, out, sa_out, sb_out, ldr_out, accumulate), note_launch();
    return cudaGetLastError();
  };
  switch (B) {
#define EPH_AXIS_ADJ_B(V) \
  case V:                 \
    return go(k_axis_adj_paired<V>);
    EPH_AXIS_ADJ_B(1) EPH_AXIS_ADJ_B(3) EPH_AXIS_ADJ_B(5) EPH_AXIS_ADJ_B(7) EPH_AXIS_ADJ_B(9) EPH_AXIS_ADJ_B(11)
    EPH_AXIS_ADJ_B(13) EPH_AXIS_ADJ_B(15) EPH_AXIS_ADJ_B(17) EPH_AXIS_ADJ_B(19) EPH_AXIS_ADJ_B(21)
    EPH_AXIS_ADJ_B(23) EPH_AXIS_ADJ_B(25) EPH_AXIS_ADJ_B(27) EPH_AXIS_ADJ_B(29) EPH_AXIS_ADJ_B(31)
    EPH_AXIS_ADJ_B(33)
#undef EPH_AXIS_ADJ_B
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_axis_adj(const double2* in, long sa_in, long sj_in, long ldr_in, int A, int R, int CC, int B,
                            const double2* E, int j0, int nj, double2* out, long sa_out, long sb_out, long ldr_out,
                            int accumulate, cudaStream_t st) {
  if (A <= 0 || R <= 0 || CC <= 0 || nj <= 0) return cudaSuccess;
  if (B < 1 || B > 33 || (B & 1) == 0 || A > 65535 || j0 < 0) return cudaErrorInvalidValue;
  const size_t smem = (size_t)nj * B * sizeof(double2);
  if (smem > 160 * 1024) return cudaErrorInvalidValue;
  const long cols = (long)R * CC;
  const dim3 grid((unsigned)((cols + 255) / 256), (unsigned)A, 1);
  auto go = [&](auto kern) -> cudaError_t {
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    kern<<<grid, 256, smem, st>>>(in, sa_in, sj_in, ldr_in, R, CC, E, j0, nj, out, sa_out, sb_out, ldr_out,
                                  accumulate), note_launch();
    return cudaGetLastError();
  };
  switch (B) {
#define EPH_AXIS_ADJ_B(V) \
  case V:                 \
    return go(k_axis_adj<V>);
    EPH_AXIS_ADJ_B(1) EPH_AXIS_ADJ_B(3) EPH_AXIS_ADJ_B(5) EPH_AXIS_ADJ_B(7) EPH_AXIS_ADJ_B(9) EPH_AXIS_ADJ_B(11)
    EPH_AXIS_ADJ_B(13) EPH_AXIS_ADJ_B(15) EPH_AXIS_ADJ_B(17) EPH_AXIS_ADJ_B(19) EPH_AXIS_ADJ_B(21)
    EPH_AXIS_ADJ_B(23) EPH_AXIS_ADJ_B(25) EPH_AXIS_ADJ_B(27) EPH_AXIS_ADJ_B(29) EPH_AXIS_ADJ_B(31)
    EPH_AXIS_ADJ_B(33)
#undef EPH_AXIS_ADJ_B
    default:
      return cudaErrorInvalidValue;
  }
}

// The adjoint of the box scatter: G[q][e][c] = w_e Sbox[q][box[e]][c] (w = NULL: 1).
__global__ void k_box_gather(const double2* __restrict__ Sbox, long sBq, int ncols, const int* __restrict__ box,
                             const double* __restrict__ we, int ne, double2* __restrict__ G, long sGq, int nq) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long per_q = (long)ne * ncols;
  if (idx >= per_q * nq) return;
  const int q = (int)(idx / per_q);
  const long rem = idx - (long)q * per_q;
  const int e = (int)(rem / ncols);
  const int c = (int)(rem - (long)e * ncols);
  const double2 v = Sbox[q * sBq + (long)box[e] * ncols + c];
  const double w = we ? we[e] : 1.0;
  G[q * sGq + rem] = make_double2(w * v.x, w * v.y);
}

cudaError_t launch_box_gather(const double2* Sbox, long sBq, int ncols, const int* box, const double* we, int ne,
                              double2* G, long sGq, int nq, cudaStream_t st) {
  const long total = (long)nq * ne * ncols;
  if (total <= 0) return cudaSuccess;
  k_box_gather<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(Sbox, sBq, ncols, box, we, ne, G, sGq, nq), note_launch();
  return cudaGetLastError();
}

// kpts[(j1 n2 + j2) n3 + j3] = (j1/n1 + s1, j2/n2 + s2, j3/n3 + s3)
__global__ void k_grid_points(int n1, int n2, int n3, double s1, double s2, double s3, double* __restrict__ k) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long nk = (long)n1 * n2 * n3;
  if (idx >= nk) return;
  const int j3 = (int)(idx % n3);
  const long r = idx / n3;
  const int j2 = (int)(r % n2);
  const int j1 = (int)(r / n2);
  k[3 * idx] = (double)j1 / (double)n1 + s1;
  k[3 * idx + 1] = (double)j2 / (double)n2 + s2;
  k[3 * idx + 2] = (double)j3 / (double)n3 + s3;
}

cudaError_t launch_grid_points(int n1, int n2, int n3, const double* shift, double* k, cudaStream_t st) {
  const long nk = (long)n1 * n2 * n3;
  if (nk <= 0) return cudaSuccess;
  k_grid_points<<<(unsigned)((nk + 255) / 256), 256, 0, st>>>(n1, n2, n3, shift[0], shift[1], shift[2], k), note_launch();
  return cudaGetLastError();
}

}  // namespace eph
