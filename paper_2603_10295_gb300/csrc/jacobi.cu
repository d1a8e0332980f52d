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

template <typename T>
struct Cx;
template <>
struct Cx<double> {
  using T2 = double2;
  __device__ static T2 make(double x, double y) { return make_double2(x, y); }
  __device__ static double rsq(double x) { return rsqrt(x); }
};
template <>
struct Cx<float> {
  using T2 = float2;
  __device__ static T2 make(float x, float y) { return make_float2(x, y); }
  __device__ static float rsq(float x) { return rsqrtf(x); }
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
    const T r = copysign(T(2), dd) / (fabs(dd) + sqrt(fma(dd, dd, T(4) * b2)));
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

// FP32-preconditioned variant: the same sweeps first run in FP32 (64x the FP64 rate on
// GB300) to an off-diagonal norm of ~1e-6 ||A||, then the FP32 eigenvectors X are refined
// in FP64 by the Ogita-Aishima iteration (Ogita & Aishima, Japan J. Indust. Appl. Math. 35,
// 2018), written for Hermitian A with the correction split into Hermitian and
// anti-Hermitian parts:
//   R = I - X^H X,  S = X^H A X,  lam_j = S_jj / (X^H X)_jj,
//   K_ij = (S_ij + (lam_i + lam_j) R_ij / 2) / (lam_j - lam_i)  (K^H = -K, one numerator per pair),
//   X <- X (I + R/2 + K),
// which makes X unitary and A-diagonal to second order in |R/2 + K| (the quadratic step of
// Newton's method for the eigendecomposition).  The FP64 work per step is three products
// of n^3 / 2 to n^3 complex multiply-adds (the Hermitian X^H X and X^H (A X) on half of
// the pairs); the update X (R/2 + K), a small correction, runs in FP32.  lam_j plus the
// second-order shift sum_i |K_ij|^2 (lam_j - lam_i) is accurate to third order.
// A step is final once every |(R/2 + K)_ij| <= th (X then exact to th^2): th = 1e-8 for
// the FP64 eigendecomposition (two steps from FP32), 1e-4 when eigenvectors are needed to
// ~1e-8 and eigenvalues to 1e-12 ||A|| (one step).  Pairs whose first-order angle would
// exceed 1e-3 (near-degenerate relative to the FP32 accuracy) are left out of K; if such a
// pair still couples above rounding level (4e-15 ||A||_F; 1e-11 for the looser target)
// after three steps, the warp falls back to the robust sequence: two Newton-Schulz steps,
// A' = V^H A V and FP64 Jacobi sweeps to polish_tol ||A||_F with a first-order finish.
template <int NP>
__global__ void __launch_bounds__(128) k_jacobi_mixed(const double2* __restrict__ A, long sA, long lda, int n,
                                                      long batch, double* __restrict__ w, long sw,
                                                      double2* __restrict__ V, long sV, int max_sweeps,
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
#pragma unroll
  for (int r = 0; r < NP; ++r) a[r] = (valid && r < n && j < n) ? A[mat * sA + (long)r * lda + j] : make_double2(0.0, 0.0);
#pragma unroll
  for (int r = 0; r < NP; ++r)
    if (r == j) a[r].y = 0.0;
  double my2 = 0.0;
#pragma unroll
  for (int r = 0; r < NP; ++r) my2 = fma(a[r].x, a[r].x, fma(a[r].y, a[r].y, my2));
  double fro2 = 0.0;
#pragma unroll
  for (int i = 0; i < NP; ++i) fro2 += shfl_d(my2, base + i);
  // the solve runs on A scaled by a power of two to ||A||_F in [0.5, 1) (exact), which keeps
  // every FP32 quantity in range; the eigenvalues are scaled back at the end
  int fexp = 0;
  frexp(sqrt(fro2), &fexp);
  const double isc = fro2 > 0.0 ? ldexp(1.0, -fexp) : 1.0;
#pragma unroll
  for (int r = 0; r < NP; ++r) a[r] = make_double2(a[r].x * isc, a[r].y * isc);
  fro2 *= isc * isc;

  // ---- FP32 preconditioning sweeps
  double2 v[NP];
  {
    float2 vf[NP];
    float2 af[NP];
#pragma unroll
    for (int r = 0; r < NP; ++r) {
      af[r] = make_float2(d2f_i(a[r].x), d2f_i(a[r].y));
      vf[r] = make_float2(r == j ? 1.f : 0.f, 0.f);
    }
    const float fro2f = (float)fro2;
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
#pragma unroll
    for (int r = 0; r < NP; ++r) v[r] = make_double2(f2d_i(vf[r].x), f2d_i(vf[r].y));
  }

  // ---- refinement
  const bool loose = polish_tol >= 1e-13;
  const float th2f = loose ? 1e-8f : 1e-16f;  // (final |E_ij|)^2
  const float tolc2f = (float)((loose ? 1e-22 : 1.6e-29) * fro2);  // (1e-11 ||A||_F)^2, (4e-15 ||A||_F)^2
  const float thc2f = 1e-6f;  // (largest first-order angle)^2
  // A and its 3M pre-sums in shared memory (per warp; element (r, s) of group g at
  // [(r NP + s) G + g], so the groups of a warp read consecutive words): frees the registers
  // of the column copy for the refinement
  __shared__ double2 shA[4][NP * NP * G];
  __shared__ double shP[4][NP * NP * G];
  const int wib = (threadIdx.x >> 5) & 3;
  if (in_group) {
#pragma unroll
    for (int r = 0; r < NP; ++r) {
      shA[wib][(r * NP + j) * G + grp] = a[r];
      shP[wib][(r * NP + j) * G + grp] = a[r].x + a[r].y;
    }
  }
  __syncwarp();
  bool done = !valid;
  double lam = 0.0;
#pragma unroll 1
  for (int step = 0; step < 3; ++step) {
    if (__all_sync(0xffffffffu, done)) break;
    double xp[NP], xm[NP];
#pragma unroll
    for (int r = 0; r < NP; ++r) {
      xp[r] = v[r].x + v[r].y;
      xm[r] = v[r].x - v[r].y;
    }
    // w = A x_j (three multiplications per complex product)
    double2 wv[NP];
    double wp[NP];
#pragma unroll
    for (int r = 0; r < NP; ++r) {
      double t1 = 0.0, t2 = 0.0, t3 = 0.0;
#pragma unroll
      for (int s2 = 0; s2 < NP; ++s2) {
        const double2 ars = shA[wib][(r * NP + s2) * G + grp];  // A[r][s2]
        const double prs = shP[wib][(r * NP + s2) * G + grp];
        t1 = fma(ars.x, v[s2].x, t1);
        t2 = fma(ars.y, v[s2].y, t2);
        t3 = fma(prs, xp[s2], t3);
      }
      wv[r] = make_double2(t1 - t2, t3 - t1 - t2);
      wp[r] = wv[r].x + wv[r].y;
    }
    // slot d: the pair (i = j + d mod NP, j); g = x_i^H x_j, s = x_i^H w_j
    auto pair_products = [&](int src, double2& g, double2& sv) {
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
    double2 g0, s0;
    pair_products(base + j, g0, s0);
    // Rayleigh quotient of x_j: 1 / g0 = 1 + e + e^2 + e^3 with e = 1 - g0 (|e| ~ 1e-6, then
    // ~1e-12; a larger |e| leaves the step unconverged through the diagonal of R/2)
    const double e0 = 1.0 - g0.x;
    const double lt = s0.x * fma(e0, fma(e0, e0 + 1.0, 1.0), 1.0);
    // The bookkeeping of the correction runs in FP32: K, the angle tests and the eigenvalue
    // shift need ~1e-7 relative precision only.  Their inputs S_ij, G_ij and the gap
    // lam_j - lam_i are formed in FP64 (they are small differences).
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
      double2 g, sv;
      pair_products(base + i, g, sv);
      const double li = shfl_d(lt, base + i);
      const float lif = shfl_d(ltf, base + i);
      const float gap = d2f_i(lt - li);
      const float hm = 0.5f * (lif + ltf);
      const float2 gf = make_float2(d2f_i(g.x), d2f_i(g.y));
      const float2 num = make_float2(fmaf(-hm, gf.x, d2f_i(sv.x)), fmaf(-hm, gf.y, d2f_i(sv.y)));
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
      xf[r] = make_float2(d2f_i(v[r].x), d2f_i(v[r].y));
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
    if (!done) {
#pragma unroll
      for (int r = 0; r < NP; ++r) v[r] = make_double2(v[r].x + f2d_i(acc[r].x), v[r].y + f2d_i(acc[r].y));
      if (emx_g <= th2f && !unres_g) {
        done = true;
        lam = lt + f2d_i(shift);
      }
    }
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
          const double2 cs = shA[wib][(r * NP + s2) * G + grp];  // A[r][s2]
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
    w[mat * sw + rank] = lam / isc;
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
#define EPH_JM(NPV)                                                                                              \
  case NPV:                                                                                                      \
    k_jacobi_mixed<NPV><<<(unsigned)blocks, threads, 0, st>>>(A, sA, lda, n, batch, w, sw, V, sV, max_sweeps, \
                                                               polish_tol, status);                              \
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
    k_jacobi<NPV><<<(unsigned)blocks, threads, 0, st>>>(A, sA, lda, n, batch, w, sw, V, sV, max_sweeps, status); \
    break;
  switch (np) {
    EPH_JC(2) EPH_JC(4) EPH_JC(6) EPH_JC(8) EPH_JC(10) EPH_JC(12) EPH_JC(14) EPH_JC(16)
    default: return cudaErrorInvalidValue;
  }
#undef EPH_JC
  return cudaGetLastError();
}

}  // namespace eph
