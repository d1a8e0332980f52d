// Batched FP64 Hermitian eigensolver: cyclic parallel (round-robin) Jacobi.
//
// Used for H(k), H(k+q) (n = nb) and D(q) (n = nm); the eigenvectors give the
// gauges U_k of Eqs. 4-5 and the phonon eigenvectors of Eq. 2.  Jacobi is the
// method of choice here because it is accurate for near-degenerate spectra
// (its eigenvector error is eps ||A|| / gap) and maps onto a warp without any
// shared memory:
//   - a group of NP lanes (NP = n rounded up to even, NP <= 16) owns one
//     matrix; lane j keeps column j of A and of the accumulated V in registers;
//   - each round rotates NP/2 disjoint pairs (p,q) at once (circle schedule);
//     the column mix A J is a register exchange with the partner lane, the row
//     mix J^H A is local to every lane;
//   - a sweep is NP-1 rounds; sweeps stop one sweep after the off-diagonal
//     norm falls below 1e-15 ||A||_F, or at max_sweeps (then *status |= 1).
// Rotation for the Hermitian 2x2 block [[a, b],[conj b, d]] (Golub & Van Loan
// sec. 8.5, with the phase of b factored out): tau = (d - a)/(2|b|),
// t = sign(tau)/(|tau| + sqrt(1 + tau^2)), c = 1/sqrt(1 + t^2), s = t c,
// J = [[c, sigma], [-conj(sigma), c]] with sigma = s b/|b|; then
// (J^H A J)_pq = 0, a' = a - t|b|, d' = d + t|b|.  Evaluated through
// r = t/|b| (one sqrt, one division, one rsqrt per rotation).
#include "eph_kernels.cuh"

namespace eph {

namespace {

__host__ __device__ constexpr int rr_partner(int j, int r, int np) {
  // circle method: player np-1 fixed, the others rotate; pairs (r+i, r-i) mod (np-1)
  return (j == np - 1) ? r : (j == r ? np - 1 : ((2 * r - j) % (np - 1) + (np - 1)) % (np - 1));
}

__device__ __forceinline__ double shfl_d(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ double2 shfl_d2(double2 v, int src) {
  return make_double2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}
__device__ __forceinline__ float shfl_d(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ float2 shfl_d2(float2 v, int src) {
  return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// FP64 <-> FP32 conversions by integer operations: on GB300 the conversion instructions share the
// FP64 pipe, which the refinement keeps busy, while the integer pipe is idle.  d2f rounds to
// nearest (ties away); both map magnitudes outside FP32's normal range below 2^-126 to 0 (only the
// small FP32 corrections of the refinement go through them).
__device__ __forceinline__ float d2f_i(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x) + (1ULL << 28);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned e = (hi >> 20) & 0x7FFu;
  const unsigned mag = __funnelshift_l(lo, hi, 3) - (896u << 23);
  return (e > 896u && e < 1151u) ? __uint_as_float(mag | (hi & 0x80000000u)) : 0.f;
}
__device__ __forceinline__ double f2d_i(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned e = (u >> 23) & 0xFFu;
  if (e == 0u) return 0.0;
  const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7FFFFFu) >> 3);
  return __hiloint2double((int)hi, (int)(u << 29));
}

// Double-float (h + l, two FP32 words, ~2^-48 relative) for the first refinement step, which runs
// on the FP32 pipe: exact two-sum (Knuth) and the two-product of an FMA; the rn intrinsics keep
// the compiler from contracting or reassociating them.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (S, T) += a b for double-float a, b: the head product's error from an FMA, the cross terms in
// FP32 (their error and the dropped a_l b_l are below 2^-48 |a b|), the head sum's error from a
// two-sum; T collects the small parts
__device__ __forceinline__ void df_acc(float& S, float& T, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  const float t = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, __fmaf_rn(ah, bh, -p)));
  float s, e;
  two_sum(S, p, s, e);
  S = s;
  T = __fadd_rn(T, __fadd_rn(e, t));
}
// normalised (h, l) of (ah + al) + (bh + bl)
__device__ __forceinline__ float2 df_add(float ah, float al, float bh, float bl) {
  float s, e, h, l;
  two_sum(ah, bh, s, e);
  two_sum(s, __fadd_rn(e, __fadd_rn(al, bl)), h, l);
  return make_float2(h, l);
}
// split of a double into h + l (|residual| <= 2^-48 |x|; magnitudes below 2^-126 flush to 0),
// by integer and FP32 operations: h = x rounded to 24 bits (d2f_i); x - h, an integer D of at most
// 29 bits in units of x's last place (the bit patterns of x and h differ by exactly that, also
// when h rounded up to the next power of two), goes to FP32 as 2^14 D_hi + D_lo through two
// exact magic-number conversions and one rounding FMA, then takes its power of two
__device__ __forceinline__ float2 df_split(double x) {
  const float h = d2f_i(x);
  const long long b = __double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e < 949 || e >= 1151) return make_float2(h, 0.f);  // the last place of x is below FP32's range
  const long long hb = (b + (1LL << 28)) & ~((1LL << 29) - 1);
  const int D = (int)(b - hb);  // |D| <= 2^28
  const float dlo = __int_as_float(0x4B000000 | (D & 0x3FFF)) - 8388608.f;           // D mod 2^14
  const float dhi = __int_as_float(0x4B400000 + (D >> 14)) - 12582912.f;             // floor(D / 2^14)
  const float l = fmaf(dhi, 16384.f, dlo) * __int_as_float((e - 948) << 23);        // x 2^(e - 1075)
  return make_float2(h, b < 0 ? -l : l);
}
__device__ __forceinline__ float4 shfl_f4(float4 v, int src) {
  return make_float4(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src),
                     __shfl_sync(0xffffffffu, v.z, src), __shfl_sync(0xffffffffu, v.w, src));
}
template <typename T>
struct Cx;
template <>
struct Cx<double> {
  using T2 = double2;
  __device__ static T2 make(double x, double y) { return make_double2(x, y); }
  __device__ static double rsq(double x) { return rsqrt(x); }
  // 2 sign(dd) / (|dd| + sqrt(s)), s > 0
  __device__ static double rot_r(double dd, double s) { return copysign(2.0, dd) / (fabs(dd) + sqrt(s)); }
};
template <>
struct Cx<float> {
  using T2 = float2;
  __device__ static T2 make(float x, float y) { return make_float2(x, y); }
  __device__ static float rsq(float x) { return rsqrtf(x); }
  // the FP32 preconditioning only steers the sweeps (the refinement sets the accuracy): the
  // hardware reciprocal square root and division, no IEEE-rounding sequences or slow paths
  __device__ static float rot_r(float dd, float s) { return __fdividef(copysignf(2.f, dd), fabsf(dd) + s * rsqrtf(s)); }
};

// One round of the circle schedule in precision T (double for the eigensolve proper,
// float for the preconditioning sweeps of k_jacobi_mixed).
template <int NP, int R, typename T>
__device__ __forceinline__ void jacobi_round(typename Cx<T>::T2 (&a)[NP], typename Cx<T>::T2 (&v)[NP], int j, int base,
                                             T thresh2) {
  using T2 = typename Cx<T>::T2;
  const int p = rr_partner(j, R, NP);
  const bool lower = j < p;
  T d = 0;
  T2 x = Cx<T>::make(0, 0);
#pragma unroll
  for (int rho = 0; rho < NP; ++rho) {
    if (rho == j) d = a[rho].x;
    if (rho == p) x = a[rho];
  }
  const T dp = shfl_d(d, base + p);
  const T2 y = shfl_d2(x, base + p);
  const T app = lower ? d : dp;
  const T aqq = lower ? dp : d;
  const T2 bq = lower ? y : x;  // A[lo][hi]
  // r = t/|b| = 2 sign(dd) / (|dd| + sqrt(dd^2 + 4|b|^2)), dd = aqq - app: the same t as
  // sign(tau)/(|tau| + sqrt(1 + tau^2)) with tau = dd/(2|b|), without forming |b|.
  const T b2 = fma(bq.x, bq.x, bq.y * bq.y);
  T c = 1, tb = 0;  // tb = t |b| = r |b|^2
  T2 sig = Cx<T>::make(0, 0);
  if (b2 > thresh2) {
    const T dd = aqq - app;
    const T r = Cx<T>::rot_r(dd, fma(dd, dd, T(4) * b2));
    tb = r * b2;
    c = Cx<T>::rsq(fma(r * r, b2, T(1)));
    const T cr = c * r;
    sig = Cx<T>::make(cr * bq.x, cr * bq.y);
  }
  // column mix (A J, V J): lower lane: c a_p - conj(sig) a_q; upper lane: sig a_p + c a_q
  const T2 coef = lower ? Cx<T>::make(-sig.x, sig.y) : sig;
#pragma unroll
  for (int rho = 0; rho < NP; ++rho) {
    const T2 o = shfl_d2(a[rho], base + p);
    const T2 m = a[rho];
    a[rho] = Cx<T>::make(fma(c, m.x, fma(coef.x, o.x, -coef.y * o.y)), fma(c, m.y, fma(coef.x, o.y, coef.y * o.x)));
  }
#pragma unroll
  for (int rho = 0; rho < NP; ++rho) {
    const T2 o = shfl_d2(v[rho], base + p);
    const T2 m = v[rho];
    v[rho] = Cx<T>::make(fma(c, m.x, fma(coef.x, o.x, -coef.y * o.y)), fma(c, m.y, fma(coef.x, o.y, coef.y * o.x)));
  }
  // row mix (J^H A) for every pair of this round: row_lo' = c row_lo - sig row_hi,
  // row_hi' = conj(sig) row_lo + c row_hi
#pragma unroll
  for (int lo = 0; lo < NP; ++lo) {
    const int hi = rr_partner(lo, R, NP);
    if (hi > lo) {
      const T cc = shfl_d(c, base + lo);
      const T2 ss = shfl_d2(sig, base + lo);
      const T2 xl = a[lo], xh = a[hi];
      a[lo] = Cx<T>::make(fma(cc, xl.x, -fma(ss.x, xh.x, -ss.y * xh.y)), fma(cc, xl.y, -fma(ss.x, xh.y, ss.y * xh.x)));
      a[hi] = Cx<T>::make(fma(cc, xh.x, fma(ss.x, xl.x, ss.y * xl.y)), fma(cc, xh.y, fma(ss.x, xl.y, -ss.y * xl.x)));
    }
  }
  // exact values of the rotated 2x2 block
  const T nd = lower ? app - tb : aqq + tb;
#pragma unroll
  for (int rho = 0; rho < NP; ++rho) {
    if (rho == p) a[rho] = Cx<T>::make(0, 0);
    if (rho == j) a[rho] = Cx<T>::make(nd, 0);
  }
}

template <int NP, int R, typename T>
struct Sweep {
  using T2 = typename Cx<T>::T2;
  __device__ __forceinline__ static void run(T2 (&a)[NP], T2 (&v)[NP], int j, int base, T thr) {
    jacobi_round<NP, R, T>(a, v, j, base, thr);
    Sweep<NP, R + 1, T>::run(a, v, j, base, thr);
  }
};
template <int NP, typename T>
struct Sweep<NP, NP - 1, T> {
  using T2 = typename Cx<T>::T2;
  __device__ __forceinline__ static void run(T2 (&)[NP], T2 (&)[NP], int, int, T) {}
};

// Undoes the column scales of unnormalised rotations (all lanes of the warp):
// A_ij /= sqrt((1 + delta_i)(1 + delta_j)), v_j /= sqrt(1 + delta_j); delta < 1e-9, so
// 1/sqrt(1 + delta) = 1 - delta/2 + 3 delta^2/8 to rounding.
template <int NP>
__device__ __forceinline__ void unit_scale(double2 (&a)[NP], double2 (&v)[NP], int base, double& delta) {
  if (!__any_sync(0xffffffffu, delta != 0.0)) return;
  const double sc = fma(delta, fma(0.375, delta, -0.5), 1.0);
#pragma unroll
  for (int rho = 0; rho < NP; ++rho) {
    const double f = sc * shfl_d(sc, base + rho);
    a[rho] = make_double2(a[rho].x * f, a[rho].y * f);
    v[rho] = make_double2(v[rho].x * sc, v[rho].y * sc);
  }
  delta = 0.0;
}

// FP64 polish round (after preconditioning every rotation is tiny): where every pair of the
// warp has |b|^2 < 1e-11 (a_qq - a_pp)^2, the rotations are applied unnormalised, J/c with c^2 =
// 1/(1 + r^2 |b|^2): the updates lose the multiplication by c (4 instead of 6 FP64 operations
// per complex element), and r needs one reciprocal instead of a square root and a division.
// J/c is a scalar multiple of the unitary J on its 2x2 block, so A stays Hermitian and V's
// columns stay orthogonal to within the product of the scale deviations (a few 1e-11 at most)
// and later angles (< 3e-6); every lane accumulates its
// column's scale 1 + delta (delta += eps + delta eps, eps = r^2 |b|^2) and the caller divides
// it out at the end.  Otherwise the columns are brought back to unit scale and the round is
// the normalised one.
template <int NP, int R>
__device__ __forceinline__ void polish_round(double2 (&a)[NP], double2 (&v)[NP], int j, int base, double thresh2,
                                             double& delta) {
  const int p = rr_partner(j, R, NP);
  const bool lower = j < p;
  double d = 0;
  double2 x = make_double2(0, 0);
#pragma unroll
  for (int rho = 0; rho < NP; ++rho) {
    if (rho == j) d = a[rho].x;
    if (rho == p) x = a[rho];
  }
  const double dp = shfl_d(d, base + p);
  const double2 y = shfl_d2(x, base + p);
  const double app = lower ? d : dp;
  const double aqq = lower ? dp : d;
  const double2 bq = lower ? y : x;
  const double b2 = fma(bq.x, bq.x, bq.y * bq.y);
  const double dd = aqq - app;
  // tiny rotation: |b|^2 < 1e-11 dd^2, where r = 2 sign(dd) / (|dd| + sqrt(dd^2 + 4|b|^2))
  // = (1/dd)(1 - |b|^2/dd^2 + 2|b|^4/dd^4 - ...) to within 1e-21 relative from its first two terms
  const bool tiny = b2 <= thresh2 || b2 < 1e-11 * (dd * dd);
  if (__all_sync(0xffffffffu, tiny)) {
    double r = 0.0;
    if (b2 > thresh2) {
      const double rd = 1.0 / dd;
      r = rd * fma(-b2 * rd, rd, 1.0);
    }
    const double tb = r * b2, eps = r * r * b2;
    const double2 sg = make_double2(r * bq.x, r * bq.y);  // sigma / c
    const double2 coef = lower ? make_double2(-sg.x, sg.y) : sg;
#pragma unroll
    for (int rho = 0; rho < NP; ++rho) {
      const double2 o = shfl_d2(a[rho], base + p);
      const double2 m = a[rho];
      a[rho] = make_double2(fma(coef.x, o.x, fma(-coef.y, o.y, m.x)), fma(coef.x, o.y, fma(coef.y, o.x, m.y)));
    }
#pragma unroll
    for (int rho = 0; rho < NP; ++rho) {
      const double2 o = shfl_d2(v[rho], base + p);
      const double2 m = v[rho];
      v[rho] = make_double2(fma(coef.x, o.x, fma(-coef.y, o.y, m.x)), fma(coef.x, o.y, fma(coef.y, o.x, m.y)));
    }
#pragma unroll
    for (int lo = 0; lo < NP; ++lo) {
      const int hi = rr_partner(lo, R, NP);
      if (hi > lo) {
        const double2 ss = shfl_d2(sg, base + lo);
        const double2 xl = a[lo], xh = a[hi];
        a[lo] = make_double2(fma(-ss.x, xh.x, fma(ss.y, xh.y, xl.x)), fma(-ss.x, xh.y, fma(-ss.y, xh.x, xl.y)));
        a[hi] = make_double2(fma(ss.x, xl.x, fma(ss.y, xl.y, xh.x)), fma(ss.x, xl.y, fma(-ss.y, xl.x, xh.y)));
      }
    }
    const double nd = (lower ? app - tb : aqq + tb) * (1.0 + eps);
#pragma unroll
    for (int rho = 0; rho < NP; ++rho) {
      if (rho == p) a[rho] = make_double2(0, 0);
      if (rho == j) a[rho] = make_double2(nd, 0);
    }
    delta = fma(delta, eps, delta + eps);
  } else {
    // a normalised rotation may mix two columns of different scale: first bring every column
    // back to unit scale
    unit_scale<NP>(a, v, base, delta);
    jacobi_round<NP, R, double>(a, v, j, base, thresh2);
  }
}

template <int NP, int R>
struct PolishSweep {
  __device__ __forceinline__ static void run(double2 (&a)[NP], double2 (&v)[NP], int j, int base, double thr,
                                             double& delta) {
    polish_round<NP, R>(a, v, j, base, thr, delta);
    PolishSweep<NP, R + 1>::run(a, v, j, base, thr, delta);
  }
};
template <int NP>
struct PolishSweep<NP, NP - 1> {
  __device__ __forceinline__ static void run(double2 (&)[NP], double2 (&)[NP], int, int, double, double&) {}
};

// Off-diagonal squared Frobenius norm of the group's matrix (all lanes get it).
template <int NP, typename T2>
__device__ __forceinline__ auto group_off2(const T2 (&a)[NP], int j, int base) {
  decltype(a[0].x) off = 0;
#pragma unroll
  for (int r = 0; r < NP; ++r)
    if (r != j) off = fma(a[r].x, a[r].x, fma(a[r].y, a[r].y, off));
  decltype(a[0].x) tot = 0;
#pragma unroll
  for (int i = 0; i < NP; ++i) tot += shfl_d(off, base + i);
  return tot;
}

}  // namespace

template <int NP>
__global__ void __launch_bounds__(128) k_jacobi(const double2* __restrict__ A, long sA, long lda, int n, long batch,
                                                double* __restrict__ w, long sw, double2* __restrict__ V, long sV,
                                                int max_sweeps, int* __restrict__ status) {
  constexpr int G = 32 / NP;
  const int lane = threadIdx.x & 31;
  const int grp0 = lane / NP;
  const bool in_group = grp0 < G;
  const int grp = in_group ? grp0 : 0;
  const int j = in_group ? lane - grp * NP : 0;
  const int base = grp * NP;
  const long warp = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long mat = warp * G + grp;
  const bool valid = in_group && mat < batch;

  double2 a[NP], v[NP];
#pragma unroll
  for (int r = 0; r < NP; ++r) {
    a[r] = (valid && r < n && j < n) ? A[mat * sA + (long)r * lda + j] : make_double2(0.0, 0.0);
    v[r] = make_double2(r == j ? 1.0 : 0.0, 0.0);
  }
  // Hermitian part of the diagonal only (imaginary parts of a Hermitian diagonal are rounding)
#pragma unroll
  for (int r = 0; r < NP; ++r)
    if (r == j) a[r].y = 0.0;

  double my2 = 0.0;
#pragma unroll
  for (int r = 0; r < NP; ++r) my2 = fma(a[r].x, a[r].x, fma(a[r].y, a[r].y, my2));
  double fro2 = 0.0;
#pragma unroll
  for (int i = 0; i < NP; ++i) fro2 += shfl_d(my2, base + i);
  const double thresh2 = 1e-36 * fro2 + 1e-300;  // rotations with |b| below 1e-18 ||A||_F are skipped
  const double tol2 = 1e-30 * fro2;

  bool conv = !valid;
  int post = valid ? 0 : 1;
  int sweep = 0;
  while (__any_sync(0xffffffffu, !(conv && post >= 1)) && sweep < max_sweeps) {
    Sweep<NP, 0, double>::run(a, v, j, base, thresh2);
    ++sweep;
    if (conv) ++post;
    double off = 0.0;
#pragma unroll
    for (int r = 0; r < NP; ++r)
      if (r != j) off = fma(a[r].x, a[r].x, fma(a[r].y, a[r].y, off));
    double tot = 0.0;
#pragma unroll
    for (int i = 0; i < NP; ++i) tot += shfl_d(off, base + i);
    if (valid && tot <= tol2) conv = true;
  }
  if (valid && j == 0 && !conv) atomicOr(status, 1);

  // sort ascending: rank of my eigenvalue among the n real ones (ties by index)
  double lam = 0.0;
#pragma unroll
  for (int r = 0; r < NP; ++r)
    if (r == j) lam = a[r].x;
  int rank = 0;
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    const double li = shfl_d(lam, base + i);
    if (i < n && (li < lam || (li == lam && i < j))) ++rank;
  }
  if (valid && j < n) {
    w[mat * sw + rank] = lam;
    double2* out = V + mat * sV;
#pragma unroll
    for (int r = 0; r < NP; ++r)
      if (r < n) out[(long)r * n + rank] = v[r];
  }
}

// FP32-preconditioned variant, two kernels: k_jacobi_f32 runs the same sweeps in FP32 (64x the
// FP64 rate on GB300) to an off-diagonal norm of ~1e-6 ||A||; k_jacobi_mixed refines its
// eigenvectors X by the Ogita-Aishima iteration (Ogita & Aishima, Japan J. Indust. Appl. Math.
// 35, 2018), written for Hermitian A with the correction split into Hermitian and anti-Hermitian
// parts:
//   R = I - X^H X,  S = X^H A X,  lam_j = S_jj / (X^H X)_jj,
//   K_ij = (S_ij + (lam_i + lam_j) R_ij / 2) / (lam_j - lam_i)  (K^H = -K, one numerator per pair),
//   X <- X (I + R/2 + K),
// which makes X unitary and A-diagonal to second order in |R/2 + K| (the quadratic step of
// Newton's method for the eigendecomposition).  The work per step is three products of n^3 / 2
// to n^3 complex multiply-adds (A X, and the Hermitian X^H X and X^H (A X) on half of the
// pairs); the update X (R/2 + K), a small correction, runs in FP32.  lam_j plus the
// second-order shift sum_i |K_ij|^2 (lam_j - lam_i) is accurate to third order.
// The first step forms the products in double-float on the FP32 pipe (~2^-47 of the largest
// term): from the FP32 estimate it only has to reach ~1e-12.  Later steps use FP64 products,
// except for the looser target below, which stays in double-float.
// A step is final once every |(R/2 + K)_ij| <= th (X then exact to th^2): th = 1e-8 for the
// FP64 eigendecomposition, and there only after an FP64 step (a double-float step then an FP64
// step from FP32); 1e-4 when eigenvectors are needed to ~1e-8 and eigenvalues to 1e-12 ||A||
// (one double-float step).  Pairs whose first-order angle would exceed 1e-3 (near-degenerate
// relative to the FP32 accuracy) are left out of K; if such a pair still couples above rounding
// level (4e-15 ||A||_F; 1e-11 for the looser target) after three steps, the warp falls back to
// the robust sequence: two Newton-Schulz steps, A' = V^H A V and FP64 Jacobi sweeps to
// polish_tol ||A||_F with a first-order finish.
// Dynamic shared memory of k_jacobi_mixed<np> for its four warps: per warp the A entries of its
// 32 / np matrices as double2, double (3M pre-sums) and float4 (double-float split), then per lane
// np float4 + np float2 (w = A x_j of a double-float step) and np / 2 + 1 float4 (pair products).
constexpr size_t jm_smem_bytes(int np) {
  return 4 * ((size_t)np * np * (32 / np) * 40 + (size_t)np * 32 * 24 + (size_t)(np / 2 + 1) * 32 * 16);
}

// x 2^s by an exponent add (integer operations: on GB300 every FP64 instruction costs the FP64
// pipe ~64 issue slots); s = 0 returns x, otherwise zero, subnormal inputs and results below
// 2^-1022 give 0
__device__ __forceinline__ double scale2_i(double x, int s) {
  if (s == 0) return x;
  const long long b = __double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e == 0 || e + s <= 0) return 0.0;
  return __longlong_as_double(b + ((long long)s << 52));
}

// Loads the group's matrix (its Hermitian part: the diagonal's imaginary parts dropped), padded to
// NP with zeros, and scales it by 2^sexp (exact) so that its largest entry lies in [0.5, 1), which
// keeps every FP32 quantity in range; the eigenvalues are scaled back by 2^-sexp at the end.
// fro2f: ||A||_F^2 of the scaled matrix in FP32 (it only sets thresholds), in [0.25, NP^2).
// Integer and FP32 operations only.
template <int NP>
__device__ __forceinline__ void jm_load(const double2* __restrict__ A, long sA, long lda, int n, long mat, bool valid,
                                        int j, int base, double2 (&a)[NP], float& fro2f, int& sexp) {
#pragma unroll
  for (int r = 0; r < NP; ++r) a[r] = (valid && r < n && j < n) ? A[mat * sA + (long)r * lda + j] : make_double2(0.0, 0.0);
#pragma unroll
  for (int r = 0; r < NP; ++r)
    if (r == j) a[r].y = 0.0;
  int em = 0;  // largest biased exponent of the group's entries
#pragma unroll
  for (int r = 0; r < NP; ++r) {
    em = max(em, (int)((__double_as_longlong(a[r].x) >> 52) & 0x7FF));
    em = max(em, (int)((__double_as_longlong(a[r].y) >> 52) & 0x7FF));
  }
#pragma unroll
  for (int i = 0; i < NP; ++i) em = max(em, __shfl_sync(0xffffffffu, em, base + i));
  sexp = em > 0 ? 1022 - em : 0;
  float my2 = 0.f;
#pragma unroll
  for (int r = 0; r < NP; ++r) {
    a[r] = make_double2(scale2_i(a[r].x, sexp), scale2_i(a[r].y, sexp));
    const float fx = d2f_i(a[r].x), fy = d2f_i(a[r].y);
    my2 = fmaf(fx, fx, fmaf(fy, fy, my2));
  }
  fro2f = 0.f;
#pragma unroll
  for (int i = 0; i < NP; ++i) fro2f += shfl_d(my2, base + i);
}

// FP32 preconditioning of k_jacobi_mixed, a kernel of its own: cyclic Jacobi sweeps in FP32 on the
// scaled matrix until its off-diagonal norm is below 1e-6 ||A||_F (12 sweeps at most), with the
// same lane layout; writes the n x n FP32 eigenvector estimate of matrix m to T + m sT (row-major,
// unsorted).  Its small register and code footprint keeps 6 CTAs per SM busy, where the fused
// kernel ran these latency-bound sweeps at the refinement's occupancy.
template <int NP>
__global__ void __launch_bounds__(128, (NP <= 8 ? 6 : 1)) k_jacobi_f32(const double2* __restrict__ A, long sA, long lda, int n,
                                                    long batch, float2* __restrict__ T, long sT) {
  constexpr int G = 32 / NP;
  const int lane = threadIdx.x & 31;
  const int grp0 = lane / NP;
  const bool in_group = grp0 < G;
  const int grp = in_group ? grp0 : 0;
  const int j = in_group ? lane - grp * NP : 0;
  const int base = grp * NP;
  const long warp = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long mat = warp * G + grp;
  const bool valid = in_group && mat < batch;
  double2 a[NP];
  float fro2f;
  int sexp;
  jm_load<NP>(A, sA, lda, n, mat, valid, j, base, a, fro2f, sexp);
  float2 vf[NP];
  float2 af[NP];
#pragma unroll
  for (int r = 0; r < NP; ++r) {
    af[r] = make_float2(d2f_i(a[r].x), d2f_i(a[r].y));
    vf[r] = make_float2(r == j ? 1.f : 0.f, 0.f);
  }
  const float thr32 = 1e-30f * fro2f + 1e-37f;
  const float tol32 = 1e-12f * fro2f;
  bool c32 = !valid;
  int s32 = 0;
  while (__any_sync(0xffffffffu, !c32) && s32 < 12) {
    Sweep<NP, 0, float>::run(af, vf, j, base, thr32);
    ++s32;
    const float off = group_off2<NP>(af, j, base);  // shuffles: every lane takes part
    if (valid && off <= tol32) c32 = true;
  }
  if (valid && j < n) {
#pragma unroll
    for (int r = 0; r < NP; ++r)
      if (r < n) T[mat * sT + (long)r * n + j] = vf[r];
  }
}

template <int NP>
__global__ void __launch_bounds__(128) k_jacobi_mixed(const double2* __restrict__ A, long sA, long lda, int n,
                                                      long batch, double* __restrict__ w, long sw, double2* V,
                                                      long sV, const float2* T, long sT, int max_sweeps,
                                                      double polish_tol, int* __restrict__ status) {
  constexpr int G = 32 / NP;
  constexpr int H = NP / 2;
  const int lane = threadIdx.x & 31;
  const int grp0 = lane / NP;
  const bool in_group = grp0 < G;
  const int grp = in_group ? grp0 : 0;
  const int j = in_group ? lane - grp * NP : 0;
  const int base = grp * NP;
  const long warp = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long mat = warp * G + grp;
  const bool valid = in_group && mat < batch;

  double2 a[NP];
  float fro2f;
  int sexp;
  jm_load<NP>(A, sA, lda, n, mat, valid, j, base, a, fro2f, sexp);
  const double fro2 = f2d_i(fro2f);
  // the FP32 eigenvector estimate of k_jacobi_f32 (padded columns: unit vectors)
  double2 v[NP];
#pragma unroll
  for (int r = 0; r < NP; ++r) {
    float2 t = make_float2(r == j ? 1.f : 0.f, 0.f);
    if (valid && j < n) t = r < n ? T[mat * sT + (long)r * n + j] : make_float2(0.f, 0.f);
    v[r] = make_double2(f2d_i(t.x), f2d_i(t.y));
  }

  // ---- refinement
  const bool loose = polish_tol >= 1e-13;
  const float th2f = loose ? 1e-8f : 1e-16f;  // (final |E_ij|)^2
  const float tolc2f = (loose ? 1e-22f : 1.6e-29f) * fro2f;  // (1e-11 ||A||_F)^2, (4e-15 ||A||_F)^2
  const float thc2f = 1e-6f;  // (largest first-order angle)^2
  // Shared memory per warp (jm_smem_bytes): A, its 3M pre-sums and its double-float split
  // (element (r, s) of group g at [(r NP + s) G + g], so the groups of a warp read consecutive
  // words; frees the registers of the column copy for the refinement), then per lane the
  // double-float w = A x_j and w_re + w_im of a step (row r at [r 32 + lane]) and the pair
  // products of its slots (slot d at [d 32 + lane]).
  extern __shared__ __align__(16) unsigned char jm_smem[];
  constexpr int EL = NP * NP * G;
  const int wib = (threadIdx.x >> 5) & 3;
  double2* shA = reinterpret_cast<double2*>(jm_smem) + wib * EL;
  double* shP = reinterpret_cast<double*>(jm_smem + 4 * EL * 16) + wib * EL;
  float4* shD = reinterpret_cast<float4*>(jm_smem + 4 * EL * 24) + wib * EL;  // (Re h, Re l, Im h, Im l)
  float4* shW = reinterpret_cast<float4*>(jm_smem + 4 * EL * 40) + wib * NP * 32 + lane;
  float2* shWp = reinterpret_cast<float2*>(jm_smem + 4 * EL * 40 + 4 * NP * 32 * 16) + wib * NP * 32 + lane;
  float4* shGS = reinterpret_cast<float4*>(jm_smem + 4 * EL * 40 + 4 * NP * 32 * 24) + wib * (H + 1) * 32 + lane;
  if (in_group) {
#pragma unroll
    for (int r = 0; r < NP; ++r) {
      shA[(r * NP + j) * G + grp] = a[r];
      if (!loose) shP[(r * NP + j) * G + grp] = a[r].x + a[r].y;  // read by FP64 steps only
      const float2 sx = df_split(a[r].x), sy = df_split(a[r].y);
      shD[(r * NP + j) * G + grp] = make_float4(sx.x, sx.y, sy.x, sy.y);
    }
  }
  __syncwarp();
  bool done = !valid;
  double lam = 0.0;

  // The correction of one step from the products of the pairs.  slot0(gx, sx) gives the real
  // parts of x_j^H x_j and x_j^H (A x_j) in double; slot(d, src, gf, sf) gives g = x_i^H x_j and
  // s = x_i^H (A x_j) in FP32 for slot d >= 1, whose x_i the lane src holds; xhead(r) is x_j[r]
  // in FP32 and update(acc, keep) sets x_j += acc (x_j unchanged where keep).  A step may end the
  // refinement only if final_ok.
  auto correct = [&](auto&& slot0, auto&& slot, auto&& xhead, auto&& update, bool final_ok) {
    double g0x, s0x;
    slot0(g0x, s0x);
    // Rayleigh quotient of x_j: 1 / g0 = 1 + e + e^2 + e^3 with e = 1 - g0 (|e| ~ 1e-6, then
    // ~1e-12; a larger |e| leaves the step unconverged through the diagonal of R/2)
    const double e0 = 1.0 - g0x;
    const double lt = s0x * fma(e0, fma(e0, e0 + 1.0, 1.0), 1.0);
    // The bookkeeping of the correction runs in FP32: K, the angle tests and the eigenvalue
    // shift need ~1e-7 relative precision only.  Their inputs S_ij, G_ij and the gap
    // lam_j - lam_i are formed at the step's precision (they are small differences).
    const float ltf = d2f_i(lt);
    const float e0f = d2f_i(e0);
    float emx = 0.25f * e0f * e0f;  // squared bound on |E_ij|
    float shift = 0.f;
    int unres = 0;
    float2 er[NP];  // er[d] = E_{(j+d) mod NP, j}
    er[0] = make_float2(0.5f * e0f, 0.f);
    float2 hf[H], kf[H];  // slot d at index d - 1
#pragma unroll
    for (int d = 1; d <= H; ++d) {
      int i = j + d;
      if (i >= NP) i -= NP;
      float2 gf, sf;
      slot(d, base + i, gf, sf);
      const double li = shfl_d(lt, base + i);
      const float lif = shfl_d(ltf, base + i);
      const float gap = d2f_i(lt - li);
      const float hm = 0.5f * (lif + ltf);
      const float2 num = make_float2(fmaf(-hm, gf.x, sf.x), fmaf(-hm, gf.y, sf.y));
      const float n2 = fmaf(num.x, num.x, num.y * num.y);
      const bool own = !(2 * d == NP && j >= H);
      float2 K = make_float2(0.f, 0.f);
      if (n2 != 0.f) {
        if (n2 <= thc2f * (gap * gap)) {
          K = make_float2(__fdiv_rn(num.x, gap), __fdiv_rn(num.y, gap));
          if (own) shift = fmaf(fmaf(K.x, K.x, K.y * K.y), gap, shift);
        } else if (n2 > tolc2f) {
          unres = 1;
        }
      }
      const float2 hh = make_float2(-0.5f * gf.x, -0.5f * gf.y);
      // |h + K|^2 and |h - K|^2 are both <= 2 (|h|^2 + |K|^2)
      if (own) emx = fmaxf(emx, 2.f * (fmaf(hh.x, hh.x, hh.y * hh.y) + fmaf(K.x, K.x, K.y * K.y)));
      hf[d - 1] = hh;
      kf[d - 1] = K;
      if (own) er[d] = make_float2(hh.x + K.x, hh.y + K.y);
    }
    // mirrored half: lane i' = j - d holds the pair (j, i') in its slot d; E_{i'j} = conj(h - k)
#pragma unroll
    for (int d = 1; d <= H; ++d) {
      int ip = j - d;
      if (ip < 0) ip += NP;
      const float2 hq = shfl_d2(hf[d - 1], base + ip);
      const float2 kq = shfl_d2(kf[d - 1], base + ip);
      const float lq = shfl_d(ltf, base + ip);
      if (2 * d < NP || j >= H) {
        er[NP - d] = make_float2(hq.x - kq.x, -(hq.y - kq.y));
        shift = fmaf(fmaf(kq.x, kq.x, kq.y * kq.y), ltf - lq, shift);
      }
    }
    // group decisions
    float emx_g = 0.f;
    int unres_g = 0;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      emx_g = fmaxf(emx_g, shfl_d(emx, base + i));
      unres_g |= __shfl_sync(0xffffffffu, unres, base + i);
    }
    // x_j += sum_i x_i E_ij in FP32
    float2 xf[NP], acc[NP];
#pragma unroll
    for (int r = 0; r < NP; ++r) {
      xf[r] = xhead(r);
      acc[r] = make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int d = 0; d < NP; ++d) {
      int i = j + d;
      if (i >= NP) i -= NP;
      const float2 e = er[d];
#pragma unroll
      for (int r = 0; r < NP; ++r) {
        const float2 xi = shfl_d2(xf[r], base + i);
        acc[r].x = fmaf(xi.x, e.x, fmaf(-xi.y, e.y, acc[r].x));
        acc[r].y = fmaf(xi.x, e.y, fmaf(xi.y, e.x, acc[r].y));
      }
    }
    update(acc, done);
    if (!done) {
      if (final_ok && emx_g <= th2f && !unres_g) {
        done = true;
        lam = lt + f2d_i(shift);
      }
    }
  };

  // FP64 products: w = A x_j with three multiplications per complex product, then the pairs
  auto step64 = [&]() {
    double xp[NP], xm[NP];
#pragma unroll
    for (int r = 0; r < NP; ++r) {
      xp[r] = v[r].x + v[r].y;
      xm[r] = v[r].x - v[r].y;
    }
    double2 wv[NP];
    double wp[NP];
#pragma unroll
    for (int r = 0; r < NP; ++r) {
      double t1 = 0.0, t2 = 0.0, t3 = 0.0;
#pragma unroll
      for (int s2 = 0; s2 < NP; ++s2) {
        const double2 ars = shA[(r * NP + s2) * G + grp];  // A[r][s2]
        const double prs = shP[(r * NP + s2) * G + grp];
        t1 = fma(ars.x, v[s2].x, t1);
        t2 = fma(ars.y, v[s2].y, t2);
        t3 = fma(prs, xp[s2], t3);
      }
      wv[r] = make_double2(t1 - t2, t3 - t1 - t2);
      wp[r] = wv[r].x + wv[r].y;
    }
    // g = x_i^H x_j, s = x_i^H w_j for the lane src holding x_i
    auto pair = [&](int src, double2& g, double2& sv) {
      double g1 = 0.0, g2 = 0.0, g3 = 0.0, s1 = 0.0, s2v = 0.0, s3 = 0.0;
#pragma unroll
      for (int r = 0; r < NP; ++r) {
        const double2 xi = shfl_d2(v[r], src);
        const double mi = shfl_d(xm[r], src);
        g1 = fma(xi.x, v[r].x, g1);
        g2 = fma(xi.y, v[r].y, g2);
        g3 = fma(mi, xp[r], g3);
        s1 = fma(xi.x, wv[r].x, s1);
        s2v = fma(xi.y, wv[r].y, s2v);
        s3 = fma(mi, wp[r], s3);
      }
      g = make_double2(g1 + g2, g3 - g1 + g2);
      sv = make_double2(s1 + s2v, s3 - s1 + s2v);
    };
    auto slot0 = [&](double& gx, double& sx) {
      double2 g, sv;
      pair(base + j, g, sv);
      gx = g.x;
      sx = sv.x;
    };
    auto slot = [&](int, int src, float2& gf, float2& sf) {
      double2 g, sv;
      pair(src, g, sv);
      gf = make_float2(d2f_i(g.x), d2f_i(g.y));
      sf = make_float2(d2f_i(sv.x), d2f_i(sv.y));
    };
    auto xhead = [&](int r) { return make_float2(d2f_i(v[r].x), d2f_i(v[r].y)); };
    auto update = [&](const float2(&acc)[NP], bool keep) {
      if (keep) return;
#pragma unroll
      for (int r = 0; r < NP; ++r) v[r] = make_double2(v[r].x + f2d_i(acc[r].x), v[r].y + f2d_i(acc[r].y));
    };
    correct(slot0, slot, xhead, update, true);
  };

  // Double-float products on the FP32 pipe (~2^-47 of the largest term per product sum): w = A x_j
  // with four multiplications per complex product from the split copy of A, the pairs with three.
  // x_j is split on entry and joined back before the update (a change below 2^-48 |x_j|).  Both
  // product phases are loops over rows and slots with their results in shared memory: unrolled,
  // the step's ~7,000 instructions overflow the instruction cache.
  auto step_df = [&](bool final_ok) {
    float4 vd[NP];  // (Re h, Re l, Im h, Im l)
    float2 xpd[NP], xmd[NP];
#pragma unroll
    for (int r = 0; r < NP; ++r) {
      const float2 sx = df_split(v[r].x), sy = df_split(v[r].y);
      vd[r] = make_float4(sx.x, sx.y, sy.x, sy.y);
      xpd[r] = df_add(sx.x, sx.y, sy.x, sy.y);
      xmd[r] = df_add(sx.x, sx.y, -sy.x, -sy.y);
    }
#pragma unroll 1
    for (int r = 0; r < NP; ++r) {
      float S1 = 0.f, T1 = 0.f, S2 = 0.f, T2 = 0.f, S3 = 0.f, T3 = 0.f, S4 = 0.f, T4 = 0.f;
      const float4* arow = shD + r * NP * G + grp;
#pragma unroll
      for (int s2 = 0; s2 < NP; ++s2) {
        const float4 ad = arow[s2 * G];  // A[r][s2]
        df_acc(S1, T1, ad.x, ad.y, vd[s2].x, vd[s2].y);
        df_acc(S2, T2, ad.z, ad.w, vd[s2].z, vd[s2].w);
        df_acc(S3, T3, ad.x, ad.y, vd[s2].z, vd[s2].w);
        df_acc(S4, T4, ad.z, ad.w, vd[s2].x, vd[s2].y);
      }
      const float2 wx = df_add(S1, T1, -S2, -T2), wy = df_add(S3, T3, S4, T4);
      shW[r * 32] = make_float4(wx.x, wx.y, wy.x, wy.y);
      shWp[r * 32] = df_add(wx.x, wx.y, wy.x, wy.y);
    }
    double g0x = 0.0, s0x = 0.0;
#pragma unroll 1
    for (int d = 0; d <= H; ++d) {
      int i = j + d;
      if (i >= NP) i -= NP;
      const int src = base + i;
      float G1 = 0.f, U1 = 0.f, G2 = 0.f, U2 = 0.f, G3 = 0.f, U3 = 0.f;
      float R1 = 0.f, V1 = 0.f, R2 = 0.f, V2 = 0.f, R3 = 0.f, V3 = 0.f;
#pragma unroll
      for (int r = 0; r < NP; ++r) {
        const float4 xi = shfl_f4(vd[r], src);
        const float2 mi = shfl_d2(xmd[r], src);
        const float4 wr = shW[r * 32];
        const float2 wpr = shWp[r * 32];
        df_acc(G1, U1, xi.x, xi.y, vd[r].x, vd[r].y);
        df_acc(G2, U2, xi.z, xi.w, vd[r].z, vd[r].w);
        df_acc(G3, U3, mi.x, mi.y, xpd[r].x, xpd[r].y);
        df_acc(R1, V1, xi.x, xi.y, wr.x, wr.y);
        df_acc(R2, V2, xi.z, xi.w, wr.z, wr.w);
        df_acc(R3, V3, mi.x, mi.y, wpr.x, wpr.y);
      }
      // real part p1 + p2, imaginary part p3 - (p1 - p2), each from exact head sums
      auto parts = [d](float P1, float Q1, float P2, float Q2, float P3, float Q3, float2& f, double& x) {
        float hs, he;
        two_sum(P1, P2, hs, he);
        const float rt = __fadd_rn(he, __fadd_rn(Q1, Q2));
        if (d == 0) x = f2d_i(hs) + f2d_i(rt);
        f.x = __fadd_rn(hs, rt);
        float ds, de;
        two_sum(P1, -P2, ds, de);
        const float dt = __fadd_rn(de, __fsub_rn(Q1, Q2));
        float ys, ye;
        two_sum(P3, -ds, ys, ye);
        f.y = __fadd_rn(ys, __fadd_rn(ye, __fsub_rn(Q3, dt)));
      };
      float2 gf, sf;
      double gx = 0.0, sx = 0.0;
      parts(G1, U1, G2, U2, G3, U3, gf, gx);
      parts(R1, V1, R2, V2, R3, V3, sf, sx);
      shGS[d * 32] = make_float4(gf.x, gf.y, sf.x, sf.y);
      if (d == 0) {
        g0x = gx;
        s0x = sx;
      }
    }
    auto slot0 = [&](double& gx, double& sx) {
      gx = g0x;
      sx = s0x;
    };
    auto slot = [&](int d, int, float2& gf, float2& sf) {
      const float4 q = shGS[d * 32];
      gf = make_float2(q.x, q.y);
      sf = make_float2(q.z, q.w);
    };
    auto xhead = [&](int r) { return make_float2(vd[r].x, vd[r].z); };
    // x_j = (h + l) + acc joined to double with one FP64 addition per value: (h + acc) by a two-sum,
    // its error into l
    auto update = [&](const float2(&acc)[NP], bool keep) {
      auto join = [](float h, float l, float c) {
        float s, e;
        two_sum(h, c, s, e);
        return f2d_i(s) + f2d_i(__fadd_rn(l, e));
      };
#pragma unroll
      for (int r = 0; r < NP; ++r)
        v[r] = make_double2(join(vd[r].x, vd[r].y, keep ? 0.f : acc[r].x), join(vd[r].z, vd[r].w, keep ? 0.f : acc[r].y));
    };
    correct(slot0, slot, xhead, update, final_ok);
  };

  // The first step runs in double-float (from the FP32 eigenvectors it only has to reach ~1e-12);
  // the FP64 eigendecomposition then finishes with FP64 steps, the looser target (a single step
  // as a rule) stays in double-float, whose eigenvalues are exact to ~1e-14 ||A||.
#pragma unroll 1
  for (int step = 0; step < 3; ++step) {
    if (__all_sync(0xffffffffu, done)) break;
    if (step == 0 || loose)
      step_df(loose);
    else
      step64();
  }

  if (!__all_sync(0xffffffffu, done)) {
    // ---- robust sequence for this warp, from the refined (or FP32) eigenvectors:
    // Newton-Schulz V <- V (3I - V^H V)/2 = V - V E/2, E = V^H V - I, with the Gram matrix
    // in FP64 and the small correction V E/2 at FP32 precision; A' = V^H A V; FP64 sweeps.
    float2 vf[NP];
#pragma unroll
    for (int r = 0; r < NP; ++r) vf[r] = make_float2((float)v[r].x, (float)v[r].y);
#pragma unroll 1
    for (int it = 0; it < 2; ++it) {
      float2 corr[NP];
#pragma unroll
      for (int r = 0; r < NP; ++r) corr[r] = make_float2(0.f, 0.f);
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        double2 vi[NP];
        double gx = 0.0, gy = 0.0;
#pragma unroll
        for (int r = 0; r < NP; ++r) {
          vi[r] = shfl_d2(v[r], base + i);
          gx = fma(vi[r].x, v[r].x, fma(vi[r].y, v[r].y, gx));
          gy = fma(vi[r].x, v[r].y, fma(-vi[r].y, v[r].x, gy));
        }
        if (i == j) gx -= 1.0;
        const float ex = (float)gx, ey = (float)gy;
#pragma unroll
        for (int r = 0; r < NP; ++r) {
          const float2 wq = shfl_d2(vf[r], base + i);
          corr[r].x = fmaf(wq.x, ex, fmaf(-wq.y, ey, corr[r].x));
          corr[r].y = fmaf(wq.x, ey, fmaf(wq.y, ex, corr[r].y));
        }
      }
#pragma unroll
      for (int r = 0; r < NP; ++r) {
        v[r].x -= (double)(0.5f * corr[r].x);
        v[r].y -= (double)(0.5f * corr[r].y);
      }
    }
    // A' = V^H A V: wv = A v_j (columns of A from all lanes), then A'[i][j] = v_i^H wv
    double2 ap[NP];
    {
      double2 wv[NP];
#pragma unroll
      for (int r = 0; r < NP; ++r) wv[r] = make_double2(0.0, 0.0);
#pragma unroll
      for (int s2 = 0; s2 < NP; ++s2) {
        const double2 vs = v[s2];
#pragma unroll
        for (int r = 0; r < NP; ++r) {
          const double2 cs = shA[(r * NP + s2) * G + grp];  // A[r][s2]
          wv[r].x = fma(cs.x, vs.x, fma(-cs.y, vs.y, wv[r].x));
          wv[r].y = fma(cs.x, vs.y, fma(cs.y, vs.x, wv[r].y));
        }
      }
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        double ax = 0.0, ay = 0.0;
#pragma unroll
        for (int r = 0; r < NP; ++r) {
          const double2 vi = shfl_d2(v[r], base + i);
          ax = fma(vi.x, wv[r].x, fma(vi.y, wv[r].y, ax));
          ay = fma(vi.x, wv[r].y, fma(-vi.y, wv[r].x, ay));
        }
        ap[i] = make_double2(ax, (i == j) ? 0.0 : ay);
      }
    }
    // padded columns stay exact unit vectors with zero coupling
    if (j >= n) {
#pragma unroll
      for (int r = 0; r < NP; ++r) {
        ap[r] = make_double2(0.0, 0.0);
        v[r] = make_double2(r == j ? 1.0 : 0.0, 0.0);
      }
    }
#pragma unroll
    for (int r = 0; r < NP; ++r)
      if (r >= n && j < n) ap[r] = make_double2(0.0, 0.0);

    const double thresh2 = 1e-36 * fro2 + 1e-300;
    const double tol2 = polish_tol * polish_tol * fro2;
    bool conv = !valid;
    int sweep = 0;
    double delta = 0.0;  // this column's accumulated scale 1 + delta from unnormalised rotations
    // first-order finish: once every remaining angle |A_ij / (A_jj - A_ii)| is below theta_max,
    // v_j += sum_i v_i A_ij / (A_jj - A_ii) completes the eigenvectors to theta_max^2 and
    // A_jj + sum_i |A_ij|^2 / (A_jj - A_ii) the eigenvalues to theta_max^3 ||A||.
    const double th2 = loose ? 1e-10 : 1e-16;
    for (;;) {
      if (__all_sync(0xffffffffu, conv)) break;
      if (sweep > 0 || loose) {
        unit_scale<NP>(ap, v, base, delta);
        double lj = 0.0;
#pragma unroll
        for (int r = 0; r < NP; ++r)
          if (r == j) lj = ap[r].x;
        bool small = true;
        double li[NP];
#pragma unroll
        for (int i = 0; i < NP; ++i) {
          li[i] = shfl_d(lj, base + i);
          const double gap = lj - li[i];
          const double m2 = fma(ap[i].x, ap[i].x, ap[i].y * ap[i].y);
          if (i != j && !(m2 <= th2 * (gap * gap))) small = false;
        }
        if (__all_sync(0xffffffffu, small)) {
          double2 dv[NP];
#pragma unroll
          for (int r = 0; r < NP; ++r) dv[r] = make_double2(0.0, 0.0);
          double dl = 0.0;
#pragma unroll
          for (int i = 0; i < NP; ++i) {
            const bool use = i != j && (ap[i].x != 0.0 || ap[i].y != 0.0);
            const double inv = use ? 1.0 / (lj - li[i]) : 0.0;
            const double2 x = make_double2(ap[i].x * inv, ap[i].y * inv);
            dl = fma(ap[i].x, x.x, fma(ap[i].y, x.y, dl));
#pragma unroll
            for (int r = 0; r < NP; ++r) {
              const double2 wq = shfl_d2(v[r], base + i);
              dv[r].x = fma(wq.x, x.x, fma(-wq.y, x.y, dv[r].x));
              dv[r].y = fma(wq.x, x.y, fma(wq.y, x.x, dv[r].y));
            }
          }
#pragma unroll
          for (int r = 0; r < NP; ++r) {
            v[r] = make_double2(v[r].x + dv[r].x, v[r].y + dv[r].y);
            if (r == j) ap[r].x = lj + dl;
          }
          conv = true;
          break;
        }
      }
      if (sweep >= max_sweeps) break;
      PolishSweep<NP, 0>::run(ap, v, j, base, thresh2, delta);
      ++sweep;
      const double off = group_off2<NP>(ap, j, base);  // shuffles: every lane takes part
      if (valid && off <= tol2) conv = true;
    }
    if (valid && j == 0 && !conv) atomicOr(status, 1);
    // undo the scales: column j of V carries sqrt(1 + delta), diagonal entry j carries 1 + delta
    // (delta < 1e-9: the second-order series are exact to rounding)
#pragma unroll
    for (int r = 0; r < NP; ++r)
      if (r == j) lam = ap[r].x;
    lam = fma(-lam, delta * (1.0 - delta), lam);
    const double vs = fma(delta, fma(0.375, delta, -0.5), 1.0);
#pragma unroll
    for (int r = 0; r < NP; ++r) v[r] = make_double2(v[r].x * vs, v[r].y * vs);
  }

  int rank = 0;
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    const double li = shfl_d(lam, base + i);
    if (i < n && (li < lam || (li == lam && i < j))) ++rank;
  }
  if (valid && j < n) {
    w[mat * sw + rank] = scale2_i(lam, -sexp);
    double2* out = V + mat * sV;
#pragma unroll
    for (int r = 0; r < NP; ++r)
      if (r < n) out[(long)r * n + rank] = v[r];
  }
}

cudaError_t launch_jacobi_mixed(const double2* A, long sA, long lda, int n, long batch, double* w, long sw, double2* V,
                                long sV, int max_sweeps, double polish_tol, int* status, cudaStream_t st) {
  if (batch <= 0) return cudaSuccess;
  if (n < 1 || n > 16) return cudaErrorInvalidValue;
  int np = (n + 1) & ~1;
  if (np < 2) np = 2;
  const int G = 32 / np;
  const long warps = (batch + G - 1) / G;
  const int threads = 128;
  const long blocks = (warps * 32 + threads - 1) / threads;
  if (blocks > 2147483647L) return cudaErrorInvalidConfiguration;
  // the FP32 estimate passes through V (n x n float2 inside each matrix's n x n double2), so V
  // must hold n x n per matrix and must not overlap A
  if (sV < (long)n * n) return cudaErrorInvalidValue;
  {
    const char* a0 = reinterpret_cast<const char*>(A);
    const char* a1 = reinterpret_cast<const char*>(A + (batch - 1) * sA + (long)(n - 1) * lda + n);
    const char* v0 = reinterpret_cast<const char*>(V);
    const char* v1 = reinterpret_cast<const char*>(V + (batch - 1) * sV + (long)n * n);
    if (v0 < a1 && a0 < v1) return cudaErrorInvalidValue;
  }
  float2* T = reinterpret_cast<float2*>(V);
  const long sT = 2 * sV;
  const size_t smem = jm_smem_bytes(np);
#define EPH_JM(NPV)                                                                                                  \
  case NPV:                                                                                                          \
    if (smem > 48 * 1024) {                                                                                          \
      cudaError_t e = cudaFuncSetAttribute(k_jacobi_mixed<NPV>, cudaFuncAttributeMaxDynamicSharedMemorySize,        \
                                           (int)smem);                                                               \
      if (e != cudaSuccess) return e;                                                                                \
    }                                                                                                                \
    k_jacobi_f32<NPV><<<(unsigned)blocks, threads, 0, st>>>(A, sA, lda, n, batch, T, sT), note_launch();                            \
    k_jacobi_mixed<NPV><<<(unsigned)blocks, threads, smem, st>>>(A, sA, lda, n, batch, w, sw, V, sV, T, sT,         \
                                                                  max_sweeps, polish_tol, status), note_launch();                   \
    break;
  switch (np) {
    EPH_JM(2) EPH_JM(4) EPH_JM(6) EPH_JM(8) EPH_JM(10) EPH_JM(12)
    default:  // 14, 16: the register-resident preconditioning would spill; plain FP64 sweeps
      return launch_jacobi(A, sA, lda, n, batch, w, sw, V, sV, max_sweeps, status, st);
  }
#undef EPH_JM
  return cudaGetLastError();
}

cudaError_t launch_jacobi(const double2* A, long sA, long lda, int n, long batch, double* w, long sw, double2* V,
                          long sV, int max_sweeps, int* status, cudaStream_t st) {
  if (batch <= 0) return cudaSuccess;
  if (n < 1 || n > 16) return cudaErrorInvalidValue;
  int np = (n + 1) & ~1;
  if (np < 2) np = 2;
  int G = 32 / np;
  long warps = (batch + G - 1) / G;
  int threads = 128;
  long blocks = (warps * 32 + threads - 1) / threads;
  if (blocks > 2147483647L) return cudaErrorInvalidConfiguration;
#define EPH_JC(NPV)                                                                                       \
  case NPV:                                                                                               \
    k_jacobi<NPV><<<(unsigned)blocks, threads, 0, st>>>(A, sA, lda, n, batch, w, sw, V, sV, max_sweeps, status), note_launch(); \
    break;
  switch (np) {
    EPH_JC(2) EPH_JC(4) EPH_JC(6) EPH_JC(8) EPH_JC(10) EPH_JC(12) EPH_JC(14) EPH_JC(16)
    default: return cudaErrorInvalidValue;
  }
#undef EPH_JC
  return cudaGetLastError();
}

}  // namespace eph
