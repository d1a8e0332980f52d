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

template <int NP, int R>
__device__ __forceinline__ void jacobi_round(double2 (&a)[NP], double2 (&v)[NP], int j, int base, double thresh2) {
  const int p = rr_partner(j, R, NP);
  const bool lower = j < p;
  double d = 0.0;
  double2 x = make_double2(0.0, 0.0);
#pragma unroll
  for (int rho = 0; rho < NP; ++rho) {
    if (rho == j) d = a[rho].x;
    if (rho == p) x = a[rho];
  }
  const double dp = shfl_d(d, base + p);
  const double2 y = shfl_d2(x, base + p);
  const double app = lower ? d : dp;
  const double aqq = lower ? dp : d;
  const double2 bq = lower ? y : x;  // A[lo][hi]
  // r = t/|b| = 2 sign(dd) / (|dd| + sqrt(dd^2 + 4|b|^2)), dd = aqq - app: the same t as
  // sign(tau)/(|tau| + sqrt(1 + tau^2)) with tau = dd/(2|b|), without forming |b|.
  const double b2 = fma(bq.x, bq.x, bq.y * bq.y);
  double c = 1.0, tb = 0.0;  // tb = t |b| = r |b|^2
  double2 sig = make_double2(0.0, 0.0);
  if (b2 > thresh2) {
    const double dd = aqq - app;
    const double r = copysign(2.0, dd) / (fabs(dd) + sqrt(fma(dd, dd, 4.0 * b2)));
    tb = r * b2;
    c = rsqrt(fma(r * r, b2, 1.0));
    const double cr = c * r;
    sig = make_double2(cr * bq.x, cr * bq.y);
  }
  // column mix (A J, V J): lower lane: c a_p - conj(sig) a_q; upper lane: sig a_p + c a_q
  const double2 coef = lower ? make_double2(-sig.x, sig.y) : sig;
#pragma unroll
  for (int rho = 0; rho < NP; ++rho) {
    const double2 o = shfl_d2(a[rho], base + p);
    const double2 m = a[rho];
    a[rho] = make_double2(fma(c, m.x, fma(coef.x, o.x, -coef.y * o.y)), fma(c, m.y, fma(coef.x, o.y, coef.y * o.x)));
  }
#pragma unroll
  for (int rho = 0; rho < NP; ++rho) {
    const double2 o = shfl_d2(v[rho], base + p);
    const double2 m = v[rho];
    v[rho] = make_double2(fma(c, m.x, fma(coef.x, o.x, -coef.y * o.y)), fma(c, m.y, fma(coef.x, o.y, coef.y * o.x)));
  }
  // row mix (J^H A) for every pair of this round: row_lo' = c row_lo - sig row_hi,
  // row_hi' = conj(sig) row_lo + c row_hi
#pragma unroll
  for (int lo = 0; lo < NP; ++lo) {
    const int hi = rr_partner(lo, R, NP);
    if (hi > lo) {
      const double cc = shfl_d(c, base + lo);
      const double2 ss = shfl_d2(sig, base + lo);
      const double2 xl = a[lo], xh = a[hi];
      a[lo] = make_double2(fma(cc, xl.x, -fma(ss.x, xh.x, -ss.y * xh.y)), fma(cc, xl.y, -fma(ss.x, xh.y, ss.y * xh.x)));
      a[hi] = make_double2(fma(cc, xh.x, fma(ss.x, xl.x, ss.y * xl.y)), fma(cc, xh.y, fma(ss.x, xl.y, -ss.y * xl.x)));
    }
  }
  // exact values of the rotated 2x2 block
  const double nd = lower ? app - tb : aqq + tb;
#pragma unroll
  for (int rho = 0; rho < NP; ++rho) {
    if (rho == p) a[rho] = make_double2(0.0, 0.0);
    if (rho == j) a[rho] = make_double2(nd, 0.0);
  }
}

template <int NP, int R>
struct Sweep {
  __device__ __forceinline__ static void run(double2 (&a)[NP], double2 (&v)[NP], int j, int base, double thr) {
    jacobi_round<NP, R>(a, v, j, base, thr);
    Sweep<NP, R + 1>::run(a, v, j, base, thr);
  }
};
template <int NP>
struct Sweep<NP, NP - 1> {
  __device__ __forceinline__ static void run(double2 (&)[NP], double2 (&)[NP], int, int, double) {}
};

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
    Sweep<NP, 0>::run(a, v, j, base, thresh2);
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
