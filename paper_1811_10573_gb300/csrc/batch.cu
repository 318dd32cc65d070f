// Many small order-3 decompositions in one set of launches.
//
// A batch holds n independent order-3 problems of different sizes and ranks
// (dims s0 x s1 x s2, rank R <= 64) and runs Algorithm 3 (PP-CP-ALS) on all
// of them at once: every stage of a sweep -- a first-level contraction
// (Sec. 2.5), a multi-TTV, the operator construction (Sec. 3.2.3), the PP
// correction of Eq. 3, the factorisation of Gamma^(n), the row solves, the
// Grams, the fitness (Sec. 5) and the decision of Algorithm 3 -- is one
// launch over every instance (blockIdx.y = instance).  Each instance keeps
// its own controller state on the device and takes part only in the stages
// of the sweep kind it runs (ALS, PP initialisation = operator build + PP
// sweep, PP approximated), so one captured graph is one sweep of the whole
// batch, whatever kind each instance takes.  Contractions, operators and
// corrections run in the batch's compute precision (float32 or float64);
// the normal-equation work (Gamma, its Cholesky factor, the solves, the
// Grams) in float64 for float64 batches and in double-float for float32
// batches; the fitness in float64.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/cpals.h"
#include "dfloat.cuh"
#include "internal.h"
#include "jacobi.cuh"

namespace {

using cpals::Launch;
using cpals::pinv_weights;
using cpals::sym_eig_jacobi;

__host__ __device__ inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

constexpr int kBR = 64;           // largest rank of a batch instance
constexpr int kBT = 256;          // threads of the contraction and element kernels
constexpr int kTuneStages = 4;    // contraction stages the autotuner tunes (CT_L, CT_R, CT_12, CT_02)
constexpr int kTileCfgs = 3;      // row-tile shapes: 64, 128, 32 rows
// Sweep kinds (as CPALS_SWEEP_*), the exact-fitness pass after the last
// sweep, and a finished instance.
enum Kind { K_ALS = 0, K_INIT = 1, K_PP = 2, K_EXACT = 3, K_DONE = -1 };

// Per-instance layout: sizes and offsets into the batch's two arenas (T:
// the compute precision; double: the float64 state).
struct BI {
  int s[3];
  int R;
  int splits;             // K splits of the MN-major ALS contraction
  int pad;
  int64_t x;              // X (s0 s1 s2)
  int64_t ac[3], dac[3];  // compute copies of A, dA (s_n R)
  int64_t ml, mr, krp, rhs, rhs2, part;
  int64_t op01, op02, op12, mp[3];
  int64_t a[3], ap[3], da[3];   // float64 factors (s_n R)
  int64_t S, W;           // 3 R x R each (float64)
  int64_t L, Z;           // R x R (float64)
  int64_t rn;             // 2 smax row norms
  int64_t sc;             // scalars: [0] fitness, [1] inner, [2] model, [3] ||X||^2,
                          // [8 + 2n] ||dA^(n)||^2, [9 + 2n] ||A^(n)||^2
  // double-float normal equations of float32 batches (T arena): the factor's
  // low words (its high words are the compute copy ac), A_p as high and low
  // words, S^(n) and W = L^-1 as high and low words, W^(n) = A^T dA and Z
  int64_t alo[3], aph[3], apl[3];
  int64_t shi, slo, lih, lil, wg, zf;
};

// Per-instance controller state of Algorithm 3 (device).
struct BC {
  int next;               // kind of the next sweep
  int ran;                // kind of the sweep being run
  int t;                  // sweeps done
  int in_run;             // PP sweeps of the current PP run
  int status;             // bit n: Gamma^(n) not finite; 1 << 8: non-finite fitness or
                          // factor norms; bit 16 + n: Gamma^(n) solved through Gamma^dagger
  int pad;
  double f_last, f_prev;
};

struct BParams {
  const BI* bi;
  BC* ctl;
  double eps, tol;
  int use_V, max_sweeps;
  int force;              // contraction stages run for every instance (autotuner timing only)
  int pad;
  double* ftrace;         // n x max_sweeps
  int* ktrace;
};

__device__ __forceinline__ bool runs_als(const BC& c) { return c.ran == K_ALS; }
// the mode-2 right-hand side X_(01)^T (A^(0) (.) A^(1)): ALS sweeps and the exact fitness
__device__ __forceinline__ bool runs_right(const BC& c) { return c.ran == K_ALS || c.ran == K_EXACT; }
__device__ __forceinline__ bool runs_init(const BC& c) { return c.ran == K_INIT; }
__device__ __forceinline__ bool runs_pp(const BC& c) { return c.ran == K_INIT || c.ran == K_PP; }

// ---------------------------------------------------------------- contractions
// Stage of a first-level contraction (Sec. 2.5, Sec. 3.2.3 level 2), all as
// out[b][m][r] = sum_k X[b][k][m] B[k][r] (MN-major) or
// out[m][r] = sum_k X[m][k] B[k][r] (K-major):
//   CT_L   K-major, m = (x0 x1), k = x2, B = A^(2): M^(L) for ALS instances,
//          M_p^(0,1) for instances building operators
//   CT_R   MN-major, m = x2, k = (x0 x1), B = A^(0) (.) A^(1): the ALS
//          right-hand side of mode 2, in K splits (partials)
//   CT_12  MN-major, m = (x1 x2), k = x0, B = A^(0): M_p^(1,2)
//   CT_02  batched MN-major, b = x0, k = x1, m = x2, B = A^(1): M_p^(0,2)
enum CtStage { CT_L = 0, CT_R = 1, CT_12 = 2, CT_02 = 3 };

template <typename T>
struct CtShape {
  bool act, kmajor;
  int64_t batch, K, M, splits, kchunk;
  const T* B;
  T* out;
};

template <typename T>
__device__ CtShape<T> ct_shape(int stage, const BI& b, const BC& c, T* tp, bool force) {
  CtShape<T> sh;
  const int64_t s0 = b.s[0], s1 = b.s[1], s2 = b.s[2];
  sh.batch = 1;
  sh.splits = 1;
  sh.kmajor = false;
  if (stage == CT_L) {
    sh.act = runs_als(c) || runs_init(c);
    sh.kmajor = true;
    sh.M = s0 * s1;
    sh.K = s2;
    sh.B = tp + b.ac[2];
    sh.out = tp + (runs_als(c) ? b.ml : b.op01);
  } else if (stage == CT_R) {
    sh.act = runs_right(c);
    sh.M = s2;
    sh.K = s0 * s1;
    sh.B = tp + b.krp;
    sh.out = tp + (b.splits > 1 ? b.part : b.mr);
    sh.splits = b.splits;
  } else if (stage == CT_12) {
    sh.act = runs_init(c);
    sh.M = s1 * s2;
    sh.K = s0;
    sh.B = tp + b.ac[0];
    sh.out = tp + b.op12;
  } else {
    sh.act = runs_init(c);
    sh.batch = s0;
    sh.M = s2;
    sh.K = s1;
    sh.B = tp + b.ac[1];
    sh.out = tp + b.op02;
  }
  sh.kchunk = cdiv(cdiv(sh.K, sh.splits), 16) * 16;
  sh.act = sh.act || force;
  return sh;
}

// Output tiles of BM rows x 16 NQ columns (NQ = ceil(R / 16), chosen per
// instance, so an instance pays for at most 15 padded columns), 256 threads,
// TM x NQ outputs per thread (rows tm TM + i, columns tn NQ + j, read from
// shared memory as vectors); a work unit
// is (batch entry, row tile, K split); the CTAs of an instance take its
// units in turn, those of an instance not in this stage return at once.  The
// next K tile is fetched into registers while the current one is multiplied
// from shared memory.  Three row-tile shapes (the autotuner picks one per
// stage and batch): BM = 64 (TM = 4), 128 (TM = 8) or 32 (TM = 2).
// N consecutive T from shared memory in 16- or 8-byte loads where the size
// allows (p aligned to the load size: the callers' row strides and offsets
// are multiples of it).
template <typename T, int N>
__device__ __forceinline__ void lds_vec(const T* p, T (&v)[N]) {
  if constexpr ((N * sizeof(T)) % 16 == 0) {
    constexpr int W = 16 / sizeof(T);
#pragma unroll
    for (int q = 0; q < N / W; q++) {
      const int4 x = reinterpret_cast<const int4*>(p)[q];
      memcpy(&v[q * W], &x, 16);
    }
  } else if constexpr (N * sizeof(T) == 8) {
    const int2 x = *reinterpret_cast<const int2*>(p);
    memcpy(&v[0], &x, 8);
  } else {
#pragma unroll
    for (int q = 0; q < N; q++) v[q] = p[q];
  }
}

constexpr int kXPad = 4;           // row padding of the staged X tile (keeps 16-byte row alignment)

template <typename T, int BM, int TM, int NQ, bool KM>
__device__ __forceinline__ void bgemm_units(const CtShape<T>& sh, const T* __restrict__ Xbase, int R,
                                            T (*Xs)[BM + kXPad], T (*Bs)[64]) {
  constexpr int BK = 16, BN = 16 * NQ;
  constexpr int XL = BK * BM / kBT;              // X elements a thread stages per K tile
  constexpr int BL = (BK * BN + kBT - 1) / kBT;  // B elements a thread stages per K tile
  const int64_t mtiles = cdiv(sh.M, BM);
  const int64_t units = mtiles * sh.batch * sh.splits;
  const int tid = threadIdx.x, tn = tid % 16, tm = tid / 16;
  // the (k, m) of this thread's staged X elements within a tile: K-major
  // (k = idx % 16, m = idx / 16) or MN-major (m = idx % BM, k = idx / BM)
  const int xk = KM ? tid % BK : tid / BM;
  const int xm = KM ? tid / BK : tid % BM;
  constexpr int XSTEP_M = KM ? kBT / BK : 0, XSTEP_K = KM ? 0 : kBT / BM;
  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
    const int64_t mt = u % mtiles;
    const int64_t rest = u / mtiles;
    const int64_t z = rest % sh.splits;
    const int64_t bb = rest / sh.splits;
    const int64_t m0 = mt * BM;
    const int64_t k0 = z * sh.kchunk, k1 = min(sh.K, k0 + sh.kchunk);
    const int mrem = (int)min((int64_t)BM, sh.M - m0);        // rows of this tile
    // element e sits at (xk + e XSTEP_K, xm + e XSTEP_M); its address at K
    // offset kk is Xt + kk (K-major: stride K between rows; MN-major: M)
    const T* Xt = Xbase + bb * sh.K * sh.M + (KM ? (m0 + xm) * sh.K + xk : (int64_t)xk * sh.M + m0 + xm);
    const int64_t estride = KM ? (int64_t)XSTEP_M * sh.K : (int64_t)XSTEP_K * sh.M;
    const int64_t kstride = KM ? 1 : sh.M;
    T acc[TM][NQ];
#pragma unroll
    for (int i = 0; i < TM; i++)
#pragma unroll
      for (int j = 0; j < NQ; j++) acc[i][j] = T(0);
    T xr[XL], br[BL];
    auto fetch = [&](int64_t kk) {
      const T* xp = Xt + (kk - k0) * kstride + k0 * kstride;
#pragma unroll
      for (int e = 0; e < XL; e++) {
        const bool ok = kk + xk + e * XSTEP_K < k1 && xm + e * XSTEP_M < mrem;
        xr[e] = ok ? xp[e * estride] : T(0);
      }
#pragma unroll
      for (int e = 0; e < BL; e++) {
        const int idx = tid + e * kBT;
        const int r = idx % BN, k = idx / BN;
        const int64_t gk = kk + k;
        br[e] = (idx < BK * BN && gk < k1 && r < R) ? sh.B[gk * R + r] : T(0);
      }
    };
    fetch(k0);
    for (int64_t kk = k0; kk < k1; kk += BK) {
      __syncthreads();                            // the previous tile is consumed
#pragma unroll
      for (int e = 0; e < XL; e++) Xs[xk + e * XSTEP_K][xm + e * XSTEP_M] = xr[e];
#pragma unroll
      for (int e = 0; e < BL; e++) {
        const int idx = tid + e * kBT;
        if (idx < BK * BN) Bs[idx / BN][idx % BN] = br[e];
      }
      __syncthreads();
      if (kk + BK < k1) fetch(kk + BK);
#pragma unroll
      for (int k = 0; k < BK; k++) {
        T av[TM], bv[NQ];
        lds_vec<T, TM>(&Xs[k][tm * TM], av);
        lds_vec<T, NQ>(&Bs[k][tn * NQ], bv);
#pragma unroll
        for (int i = 0; i < TM; i++)
#pragma unroll
          for (int j = 0; j < NQ; j++) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
      }
    }
    T* o = sh.out + (z * sh.batch + bb) * sh.M * R;
#pragma unroll
    for (int i = 0; i < TM; i++) {
      const int64_t m = m0 + tm * TM + i;
      if (m >= sh.M) continue;
#pragma unroll
      for (int j = 0; j < NQ; j++) {
        const int r = tn * NQ + j;
        if (r < R) o[m * R + r] = acc[i][j];
      }
    }
  }
}

template <typename T, int BM, int TM, bool KM>
__device__ __forceinline__ void bgemm_nq(const CtShape<T>& sh, const T* X, int R, T (*Xs)[BM + kXPad],
                                         T (*Bs)[64]) {
  switch ((R + 15) >> 4) {
    case 1: bgemm_units<T, BM, TM, 1, KM>(sh, X, R, Xs, Bs); break;
    case 2: bgemm_units<T, BM, TM, 2, KM>(sh, X, R, Xs, Bs); break;
    case 3: bgemm_units<T, BM, TM, 3, KM>(sh, X, R, Xs, Bs); break;
    default: bgemm_units<T, BM, TM, 4, KM>(sh, X, R, Xs, Bs); break;
  }
}

template <typename T, int BM, int TM>
__global__ void __launch_bounds__(kBT, sizeof(T) == 4 ? (BM == 32 ? 3 : 2) : 1) bgemm_kernel(BParams P, int stage, T* __restrict__ tp) {
  const BI b = P.bi[blockIdx.y];
  const BC c = P.ctl[blockIdx.y];
  const CtShape<T> sh = ct_shape<T>(stage, b, c, tp, P.force != 0);
  if (!sh.act) return;
  __shared__ __align__(16) T Xs[16][BM + kXPad];
  __shared__ __align__(16) T Bs[16][64];
  if (sh.kmajor) bgemm_nq<T, BM, TM, true>(sh, tp + b.x, b.R, Xs, Bs);
  else bgemm_nq<T, BM, TM, false>(sh, tp + b.x, b.R, Xs, Bs);
}

// M^(2) = sum of the K-split partials of CT_R in split order (ALS instances).
template <typename T>
__global__ void breduce_kernel(BParams P, T* __restrict__ tp) {
  const BI b = P.bi[blockIdx.y];
  if (!runs_right(P.ctl[blockIdx.y]) || b.splits <= 1) return;
  const int64_t n = (int64_t)b.s[2] * b.R;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    T acc = T(0);
    for (int z = 0; z < b.splits; z++) acc += tp[b.part + z * n + i];
    tp[b.mr + i] = acc;
  }
}

// Khatri-Rao product A^(0) (.) A^(1), row (x0 x1) = x0 s1 + x1 (ALS instances).
template <typename T>
__global__ void bkrp_kernel(BParams P, T* __restrict__ tp) {
  const BI b = P.bi[blockIdx.y];
  if (!runs_right(P.ctl[blockIdx.y])) return;
  const int R = b.R;
  const int64_t n = (int64_t)b.s[0] * b.s[1] * R;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(i % R);
    const int64_t row = i / R;
    const int64_t x0 = row / b.s[1], x1 = row % b.s[1];
    tp[b.krp + i] = tp[b.ac[0] + x0 * R + r] * tp[b.ac[1] + x1 * R + r];
  }
}

// Multi-TTV (Sec. 2.5 lower level): out[o][q][r] = sum_x in[o][x][q][r] A[x][r].
//   TT_ALS0  rhs = M^(L) contracted over x1 with A^(1) (mode 0, ALS)
//   TT_ALS1  rhs = M^(L) contracted over x0 with A^(0) (mode 1, ALS)
//   TT_MP    M_p^(0) = M_p^(0,1) over x1 with A^(1), M_p^(1) = M_p^(0,1)
//            over x0 with A^(0), M_p^(2) = M_p^(0,2) over x0 with A^(0)
//            (operator build; blockIdx.z picks the output)
enum TtStage { TT_ALS0 = 0, TT_ALS1 = 1, TT_MP = 2 };

template <typename T>
__global__ void bttv_kernel(BParams P, int stage, T* __restrict__ tp) {
  const BI b = P.bi[blockIdx.y];
  const BC c = P.ctl[blockIdx.y];
  const int R = b.R;
  const int64_t s0 = b.s[0], s1 = b.s[1], s2 = b.s[2];
  const T *in, *A;
  T* out;
  int64_t outer, inner;
  int sw;
  if (stage == TT_ALS0 || stage == TT_ALS1) {
    if (!runs_als(c)) return;
    in = tp + b.ml;
    out = tp + b.rhs;
    if (stage == TT_ALS0) {
      A = tp + b.ac[1]; outer = s0; sw = (int)s1; inner = 1;
    } else {
      A = tp + b.ac[0]; outer = 1; sw = (int)s0; inner = s1;
    }
  } else {
    if (!runs_init(c)) return;
    const int w = blockIdx.z;
    if (w == 0) {
      in = tp + b.op01; A = tp + b.ac[1]; out = tp + b.mp[0]; outer = s0; sw = (int)s1; inner = 1;
    } else if (w == 1) {
      in = tp + b.op01; A = tp + b.ac[0]; out = tp + b.mp[1]; outer = 1; sw = (int)s0; inner = s1;
    } else {
      in = tp + b.op02; A = tp + b.ac[0]; out = tp + b.mp[2]; outer = 1; sw = (int)s0; inner = s2;
    }
  }
  const int64_t n = outer * inner * R;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(i % R);
    const int64_t q = (i / R) % inner, o = i / (R * inner);
    const T* src = in + (o * sw * inner + q) * R + r;
    T acc = T(0);
    for (int x = 0; x < sw; x++) acc = fma(src[(int64_t)x * inner * R], A[(int64_t)x * R + r], acc);
    out[i] = acc;
  }
}

// ---------------------------------------------------------------- normal equations (float64)
// Stage selector of the per-mode kernels: the ALS sweep's update of mode n,
// or the PP sweep's (instances in PP initialisation or approximated sweeps).
// NE_INIT: the Grams and norms of the initial factors (Algorithm 3 starts
// with S^(n) = A^(n)T A^(n) and dA^(n) = A^(n)), for every instance.
// NE_SWEEP: the update of mode n in whichever sweep kind the instance runs
// (ALS: exact right-hand side, dA against the old factor; PP: Eq. 3's
// right-hand side, dA against A_p, W^(n) for the second-order terms).
enum NeStage { NE_ALS = 0, NE_PP = 1, NE_INIT = 2, NE_SWEEP = 3 };

__device__ __forceinline__ bool ne_active(int stage, const BC& c) {
  if (stage == NE_INIT) return c.ran != K_DONE;
  if (stage == NE_SWEEP) return runs_als(c) || runs_pp(c);
  return stage == NE_ALS ? runs_als(c) : runs_pp(c);
}
__device__ __forceinline__ bool ne_als(int stage, const BC& c) {
  return stage == NE_ALS || (stage == NE_SWEEP && runs_als(c));
}
__device__ __forceinline__ bool ne_pp(int stage, const BC& c) {
  return stage == NE_PP || (stage == NE_SWEEP && runs_pp(c));
}

// Gamma^(n) = S^(a) * S^(b) (the other two modes' Grams, Algorithm 1), its
// Cholesky factor L (right-looking, in shared memory) and W = L^-1 (written
// in place of L: the row solves use W alone), and for PP sweeps with
// the second-order terms Z = W^(a) * W^(b) (Eq. 3 for order 3: the one pair
// {a, b}, W^(i) = A^(i)T dA^(i)), so that V^(n,a,b) = A^(n) Z.  One CTA per
// instance; a non-positive pivot sets bit n of the instance's status.
__global__ void __launch_bounds__(128) bchol_kernel(BParams P, int stage, int n, double* __restrict__ dp) {
  BC& cc = P.ctl[blockIdx.y];
  const BI b = P.bi[blockIdx.y];
  if (!ne_active(stage, cc)) return;
  const int R = b.R, RS = kBR + 1;
  const int a0 = n == 0 ? 1 : 0, a1 = n == 2 ? 1 : 2;
  const double* S = dp + b.S;
  const double* W = dp + b.W;
  __shared__ double G[kBR * (kBR + 1)];
  __shared__ double il_sh;
  __shared__ int bad;
  const bool v = ne_pp(stage, cc) && P.use_V;
  for (int idx = threadIdx.x; idx < R * R; idx += blockDim.x) {
    const int i = idx / R, j = idx % R;
    G[i * RS + j] = S[a0 * R * R + idx] * S[a1 * R * R + idx];
    if (v) dp[b.Z + idx] = W[a0 * R * R + idx] * W[a1 * R * R + idx];
  }
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int k = 0; k < R; k++) {
    if (threadIdx.x == 0) {
      const double piv = G[k * RS + k];
      if (!(piv > 0.0) || !isfinite(piv)) {
        bad = 1;
      } else {
        const double il = rsqrt(piv);
        il_sh = il;
        G[k * RS + k] = piv * il;
      }
    }
    __syncthreads();
    if (bad) break;
    const double il = il_sh;
    for (int i = k + 1 + threadIdx.x; i < R; i += blockDim.x) G[i * RS + k] *= il;
    __syncthreads();
    // trailing update of the lower triangle: one warp per row, lanes over columns
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = k + 1 + warp; i < R; i += nw) {
      const double lik = G[i * RS + k];
      for (int j = k + 1 + lane; j <= i; j += 32) G[i * RS + j] = fma(-lik, G[j * RS + k], G[i * RS + j]);
    }
    __syncthreads();
  }
  if (bad) {
    // not positive definite: Gamma = V diag(w) V^T (cyclic Jacobi) and the
    // dense factor W = diag(w^+)^(1/2) V^T in place of L^-1, so that the
    // solve's W^T W is Algorithm 1's Gamma^dagger (status bit 16 + n); V is
    // accumulated in the factor's own storage.  A non-finite Gamma is an
    // error (bit n).
    __shared__ double wq[kBR];
    double* V = dp + b.L;
    int fin = 1;
    for (int idx = threadIdx.x; idx < R * R; idx += blockDim.x) {
      const int i = idx / R, j = idx % R;
      const double g = S[a0 * R * R + idx] * S[a1 * R * R + idx];
      G[i * RS + j] = g;
      V[idx] = i == j ? 1.0 : 0.0;
      fin &= isfinite(g) ? 1 : 0;
    }
    if (!__syncthreads_and(fin)) {
      if (threadIdx.x == 0) atomicOr(&cc.status, 1 << n);
      return;
    }
    sym_eig_jacobi(G, RS, V, R, R);
    pinv_weights(G, RS, R, true, wq);
    for (int idx = threadIdx.x; idx < R * R; idx += blockDim.x) {
      const int k = idx / R, c = idx % R;
      G[k * RS + c] = wq[k] * V[c * R + k];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < R * R; idx += blockDim.x) V[idx] = G[(idx / R) * RS + idx % R];
    if (threadIdx.x == 0) atomicOr(&cc.status, 1 << (16 + n));
    return;
  }
  if (threadIdx.x == 0 && ((cc.status >> (16 + n)) & 1)) atomicAnd(&cc.status, ~(1 << (16 + n)));
  // W = L^-1 (lower triangular), row by row: W[k] = V[k] / L[k][k] with
  // V[i] = e_i - sum_{k<i} L[i][k] W[k] (right-looking: row k of V is final
  // at step k and updates the rows below it).  V[i][c] (c <= i) lives in the
  // unused upper part of G at G[c][i + 1]; dinv[k] = 1 / L[k][k].
  __shared__ double dinv[kBR];
  for (int i = threadIdx.x; i < R; i += blockDim.x) dinv[i] = 1.0 / G[i * RS + i];
  for (int idx = threadIdx.x; idx < R * R; idx += blockDim.x) {
    const int i = idx / R, c = idx % R;
    if (c <= i) G[c * RS + i + 1] = i == c ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int k = 0; k + 1 < R; k++) {
    const int w = k + 1, cnt = (R - k - 1) * w;
    const double dk = dinv[k];
    for (int idx = threadIdx.x; idx < cnt; idx += blockDim.x) {
      const int i = k + 1 + idx / w, c = idx % w;
      G[c * RS + i + 1] = fma(-G[i * RS + k] * dk, G[c * RS + k + 1], G[c * RS + i + 1]);
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < R * R; idx += blockDim.x) {
    const int i = idx / R, c = idx % R;
    dp[b.L + idx] = c <= i ? G[c * RS + i + 1] * dinv[i] : 0.0;
  }
}

// Row solves of mode n: a Gamma = b with b = rhs (+ A_old Z for the PP
// second-order terms, formed in the compute precision T), through
// Gamma^-1 = W^T W (W = L^-1 from the factorisation): u = b W^T, a = u W, so
// every output is an independent dot product and no row runs a chain of R
// dependent steps.  Then the new factor, dA^(n) = A_new - A_old (ALS) or
// A_new - A_p (PP), the compute copies and the per-row ||dA||^2, ||A_new||^2.
// The PP sweep's last mode also keeps its full right-hand side (rhs2) for the
// fitness estimate.  A mode whose factorisation failed keeps its factor.
// kSolveCtas CTAs of 256 threads per instance, each with its own copy of W
// (and Z) in shared memory, take tiles of kSolveTR rows in turn; a row's 16
// threads hold outputs r = l, l + 16, l + 32, l + 48.
constexpr int kSolveCtas = 4;
constexpr int kSolveTR = 16;

template <typename T>
constexpr size_t bsolve_smem() {
  return (size_t)kBR * (kBR + 1) * (sizeof(double) + sizeof(T)) + 2 * (size_t)kSolveTR * (kBR + 1) * sizeof(double);
}

template <typename T>
__global__ void __launch_bounds__(256) bsolve_kernel(BParams P, int stage, int n, T* __restrict__ tp,
                                                     double* __restrict__ dp) {
  const BI& b = P.bi[blockIdx.y];   // fields read once, indexed by mode
  const BC c = P.ctl[blockIdx.y];
  if (!ne_active(stage, c)) return;
  const int R = b.R, s = b.s[n], RS = kBR + 1;
  const bool failed = (c.status >> n) & 1;
  const bool dense = (c.status >> (16 + n)) & 1;   // W from Gamma^dagger: no zero triangle
  const bool als = ne_als(stage, c);
  const bool v = ne_pp(stage, c) && P.use_V;
  extern __shared__ __align__(16) unsigned char bs_raw[];
  double* Ws = reinterpret_cast<double*>(bs_raw);              // W[j][k], k <= j unless dense
  double* bt = Ws + kBR * RS;                                   // b of the tile's rows
  double* ut = bt + kSolveTR * RS;                              // u = b W^T
  T* Zs = reinterpret_cast<T*>(ut + kSolveTR * RS);             // Z in T
  if (!failed) {
    for (int idx = threadIdx.x; idx < R * R; idx += blockDim.x) {
      Ws[(idx / R) * RS + idx % R] = dp[b.L + idx];
      if (v) Zs[(idx / R) * RS + idx % R] = (T)dp[b.Z + idx];
    }
  }
  const T* rhs = tp + (als && n == 2 ? b.mr : b.rhs);
  const T* Ac = tp + b.ac[n];                   // compute copy of the factor before the update
  double* A = dp + b.a[n];
  const double* ref = dp + (als ? b.a[n] : b.ap[n]);
  double* dA = dp + b.da[n];
  T* Anew_c = tp + b.ac[n];
  T* dA_c = tp + b.dac[n];
  T* rhs2 = tp + b.rhs2;
  double* rn = dp + b.rn;
  const int t = threadIdx.x >> 4, l = threadIdx.x & 15;
  const int nq = (R + 15) >> 4;                 // 16-column chunks in use (block-uniform)
  for (int y0 = blockIdx.x * kSolveTR; y0 < s; y0 += gridDim.x * kSolveTR) {
    const int y = y0 + t;
    const bool on = y < s;
    __syncthreads();                            // W, Z staged; the previous tile's bt/ut consumed
    if (!failed) {
      // b = rhs + A_old Z
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const int r = l + 16 * q;
        if (q >= nq || r >= R) continue;
        double bv = on ? (double)rhs[(int64_t)y * R + r] : 0.0;
        if (v && on) {
          T acc = T(0);
          const T* ar = Ac + (int64_t)y * R;
          for (int k = 0; k < R; k++) acc = fma(ar[k], Zs[k * RS + r], acc);
          bv += (double)acc;
          if (n == 2) rhs2[(int64_t)y * R + r] = (T)bv;
        }
        bt[t * RS + r] = bv;
      }
    }
    __syncthreads();
    if (!failed) {
      // u_j = sum_{k <= j} b_k W[j][k]
#pragma unroll
      for (int q = 0; q < 4; q++) {
        if (q >= nq) break;
        const int j = l + 16 * q;
        const int kend = dense ? R - 1 : min(16 * q + 15, R - 1);   // warp-uniform trip count
        double u = 0.0;
        for (int k = 0; k <= kend; k++)
          if (dense || k <= j) u = fma(bt[t * RS + k], Ws[j * RS + k], u);
        if (j < R) ut[t * RS + j] = u;
      }
    }
    __syncthreads();
    double av[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
      av[q] = 0.0;
      if (q >= nq || failed) continue;
      // a_r = sum_{j >= r} u_j W[j][r]
      const int r = l + 16 * q;
      double a = 0.0;
      for (int j = dense ? 0 : 16 * q; j < R; j++)
        if (dense || j >= r) a = fma(ut[t * RS + j], Ws[j * RS + r], a);
      av[q] = a;
    }
    double nd = 0.0, na = 0.0;
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int r = l + 16 * q;
      if (q >= nq || r >= R || !on) continue;
      const int64_t o = (int64_t)y * R + r;
      const double old = A[o];
      const double an = failed ? old : av[q];
      const double d = failed ? dA[o] : an - (als ? old : ref[o]);
      A[o] = an;
      dA[o] = d;
      Anew_c[o] = (T)an;
      dA_c[o] = (T)d;
      nd = fma(d, d, nd);
      na = fma(an, an, na);
    }
#pragma unroll
    for (int off = 8; off > 0; off >>= 1) {
      nd += __shfl_xor_sync(0xffffffffu, nd, off);
      na += __shfl_xor_sync(0xffffffffu, na, off);
    }
    if (l == 0 && on) {
      rn[2 * y] = nd;
      rn[2 * y + 1] = na;
    }
  }
}

// Grams of mode n after its update: S^(n) = A^T A (float64, both triangles)
// and, in PP sweeps, W^(n) = A^T dA (in the compute precision: it only feeds
// the second-order terms), in 32 x 32 output blocks, one CTA per block: the
// lower-triangle blocks of S (1 or 3) and the blocks of W^(n) (1 or 4).  A
// block's 256 threads hold 2 x 2 outputs each and stream the rows through
// shared memory in chunks of 32; every entry is one dot product over the
// rows in row order.  CTA 0 also sums the row norms into ||dA^(n)||^2 and
// ||A^(n)||^2.
constexpr int kGramCtas = 7;

template <typename U>
__device__ void gram_block(const U* __restrict__ X, const U* __restrict__ Y, int s, int R, int i0, int j0,
                           U* xs, U* ys, U (&acc)[2][2]) {
  const int ti = threadIdx.x >> 4, tj = threadIdx.x & 15;
#pragma unroll
  for (int a = 0; a < 2; a++)
#pragma unroll
    for (int c = 0; c < 2; c++) acc[a][c] = U(0);
  for (int y0 = 0; y0 < s; y0 += 32) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < 32 * 32; idx += blockDim.x) {
      const int yy = idx >> 5, cc = idx & 31, y = y0 + yy;
      xs[yy * 33 + cc] = (y < s && i0 + cc < R) ? X[(int64_t)y * R + i0 + cc] : U(0);
      ys[yy * 33 + cc] = (y < s && j0 + cc < R) ? Y[(int64_t)y * R + j0 + cc] : U(0);
    }
    __syncthreads();
    const int ye = min(32, s - y0);
    for (int yy = 0; yy < ye; yy++) {
      const U x0 = xs[yy * 33 + ti], x1 = xs[yy * 33 + ti + 16];
      const U z0 = ys[yy * 33 + tj], z1 = ys[yy * 33 + tj + 16];
      acc[0][0] = fma(x0, z0, acc[0][0]);
      acc[0][1] = fma(x0, z1, acc[0][1]);
      acc[1][0] = fma(x1, z0, acc[1][0]);
      acc[1][1] = fma(x1, z1, acc[1][1]);
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) bgram_kernel(BParams P, int stage, int n, T* __restrict__ tp,
                                                    double* __restrict__ dp) {
  const BI& b = P.bi[blockIdx.y];   // fields read once, indexed by mode
  const BC c = P.ctl[blockIdx.y];
  if (!ne_active(stage, c)) return;
  const int R = b.R, s = b.s[n];
  const int nb = (R + 31) >> 5;                 // 1 or 2 blocks per side (R <= 64)
  const int nS = nb * (nb + 1) / 2;
  const int nW = ne_pp(stage, c) ? nb * nb : 0;
  const int blk = blockIdx.x;
  __shared__ double gs[2 * 32 * 33];
  const int ti = threadIdx.x >> 4, tj = threadIdx.x & 15;
  if (blk < nS) {
    // lower-triangle blocks (0,0), (1,0), (1,1)
    const int bi = blk >= 1, bj = blk == 2;
    const int i0 = 32 * bi, j0 = 32 * bj;
    double acc[2][2];
    const double* A = dp + b.a[n];
    gram_block<double>(A, A, s, R, i0, j0, gs, gs + 32 * 33, acc);
    double* S = dp + b.S + (int64_t)n * R * R;
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
      for (int e = 0; e < 2; e++) {
        const int i = i0 + ti + 16 * a, j = j0 + tj + 16 * e;
        if (i < R && j < R) {
          S[i * R + j] = acc[a][e];
          if (bi != bj) S[j * R + i] = acc[a][e];
        }
      }
  } else if (blk < nS + nW) {
    const int f = blk - nS, i0 = 32 * (f / nb), j0 = 32 * (f % nb);
    T acc[2][2];
    T* gt = reinterpret_cast<T*>(gs);
    gram_block<T>(tp + b.ac[n], tp + b.dac[n], s, R, i0, j0, gt, gt + 32 * 33, acc);
    double* Wn = dp + b.W + (int64_t)n * R * R;
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
      for (int e = 0; e < 2; e++) {
        const int i = i0 + ti + 16 * a, j = j0 + tj + 16 * e;
        if (i < R && j < R) Wn[i * R + j] = (double)acc[a][e];
      }
  }
  if (blk != 0) return;
  __shared__ double rd[256], ra[256];
  double x = 0.0, z = 0.0;
  const double* A = dp + b.a[n];
  if (stage == NE_INIT) {
    for (int64_t e = threadIdx.x; e < (int64_t)s * R; e += blockDim.x) z = fma(A[e], A[e], z);
    x = z;
  } else {
    for (int y = threadIdx.x; y < s; y += blockDim.x) {
      x += dp[b.rn + 2 * y];
      z += dp[b.rn + 2 * y + 1];
    }
  }
  rd[threadIdx.x] = x;
  ra[threadIdx.x] = z;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) {
      rd[threadIdx.x] += rd[threadIdx.x + st];
      ra[threadIdx.x] += ra[threadIdx.x + st];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    dp[b.sc + 8 + 2 * n] = rd[0];
    dp[b.sc + 9 + 2 * n] = ra[0];
  }
}

// ---------------------------------------------------------------- normal equations (double-float)
// Float32 batches run the normal-equation stages in double-float arithmetic
// (hi + lo pairs of floats, 48-bit significand; dfloat.cuh) on the float32
// pipes, as the float32 contexts do: GB300's float64 pipe runs at 1/64 of the
// float32 rate.  Same stages, orders and layout as the float64 kernels above;
// the float64 factor and Grams are still written (high + low words) for the
// fitness, the PP set-up and the host.
using namespace cpals::dfa;

// Gamma^(n) = S^(a) * S^(b), its Cholesky factor and W = L^-1 (lower, in the
// unused upper part of G as in the float64 kernel), all double-float; Z =
// W^(a) * W^(b) in float for the second-order terms.  1 / L[k][k] is the
// pivot's reciprocal square root, taken once.
__global__ void __launch_bounds__(256) bchol_df_kernel(BParams P, int stage, int n, float* __restrict__ tp,
                                                       double* __restrict__ dp) {
  BC& cc = P.ctl[blockIdx.y];
  const BI& b = P.bi[blockIdx.y];
  if (!ne_active(stage, cc)) return;
  const int R = b.R, RS = kBR + 1, RR = R * R;
  const int a0 = n == 0 ? 1 : 0, a1 = n == 2 ? 1 : 2;
  const float* sh = tp + b.shi;
  const float* sl = tp + b.slo;
  const float* wg = tp + b.wg;
  float* zf = tp + b.zf;
  __shared__ float2 G[kBR * (kBR + 1)];
  __shared__ float2 dinv[kBR];
  __shared__ int bad;
  const bool v = ne_pp(stage, cc) && P.use_V;
  for (int idx = threadIdx.x; idx < RR; idx += blockDim.x) {
    const int i = idx / R, j = idx % R;
    const dfl x{sh[a0 * RR + idx], sl[a0 * RR + idx]}, y{sh[a1 * RR + idx], sl[a1 * RR + idx]};
    G[i * RS + j] = pk(df_mul(x, y));
    if (v) zf[idx] = wg[a0 * RR + idx] * wg[a1 * RR + idx];
  }
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int k = 0; k < R; k++) {
    if (threadIdx.x == 0) {
      const dfl piv = upk(G[k * RS + k]);
      if (!(piv.hi > 0.f) || !isfinite(piv.hi)) {
        bad = 1;
      } else {
        const dfl il = df_rsqrt(piv);
        dinv[k] = pk(il);
        G[k * RS + k] = pk(df_mul(piv, il));
      }
    }
    __syncthreads();
    if (bad) break;
    const dfl il = upk(dinv[k]);
    for (int i = k + 1 + threadIdx.x; i < R; i += blockDim.x) G[i * RS + k] = pk(df_mul(upk(G[i * RS + k]), il));
    __syncthreads();
    for (int i = k + 1 + warp; i < R; i += nw) {
      const dfl lik = upk(G[i * RS + k]);
      for (int j = k + 1 + lane; j <= i; j += 32)
        G[i * RS + j] = pk(df_sub(upk(G[i * RS + j]), df_mul(lik, upk(G[j * RS + k]))));
    }
    __syncthreads();
  }
  if (bad) {
    // not positive definite: the dense factor W = diag(w^+)^(1/2) V^T of
    // Gamma^dagger as in the float64 kernel, from Gamma in float64 (G's
    // storage reused), V in the float64 scratch dp[b.L]; written as
    // double-float (status bit 16 + n)
    __shared__ double wq[kBR];
    double* Gd = reinterpret_cast<double*>(G);
    double* V = dp + b.L;
    int fin = 1;
    for (int idx = threadIdx.x; idx < RR; idx += blockDim.x) {
      const int i = idx / R, j = idx % R;
      const double g = ((double)sh[a0 * RR + idx] + (double)sl[a0 * RR + idx]) *
                       ((double)sh[a1 * RR + idx] + (double)sl[a1 * RR + idx]);
      Gd[i * RS + j] = g;
      V[idx] = i == j ? 1.0 : 0.0;
      fin &= isfinite(g) ? 1 : 0;
    }
    if (!__syncthreads_and(fin)) {
      if (threadIdx.x == 0) atomicOr(&cc.status, 1 << n);
      return;
    }
    sym_eig_jacobi(Gd, RS, V, R, R);
    pinv_weights(Gd, RS, R, true, wq);
    for (int idx = threadIdx.x; idx < RR; idx += blockDim.x) {
      const int k = idx / R, c = idx % R;
      const dfl f = df_of(wq[k] * V[c * R + k]);
      tp[b.lih + idx] = f.hi;
      tp[b.lil + idx] = f.lo;
    }
    if (threadIdx.x == 0) atomicOr(&cc.status, 1 << (16 + n));
    return;
  }
  if (threadIdx.x == 0 && ((cc.status >> (16 + n)) & 1)) atomicAnd(&cc.status, ~(1 << (16 + n)));
  for (int idx = threadIdx.x; idx < RR; idx += blockDim.x) {
    const int i = idx / R, c = idx % R;
    if (c <= i) G[c * RS + i + 1] = make_float2(i == c ? 1.f : 0.f, 0.f);
  }
  __syncthreads();
  for (int k = 0; k + 1 < R; k++) {
    const int w = k + 1, cnt = (R - k - 1) * w;
    const dfl dk = upk(dinv[k]);
    for (int idx = threadIdx.x; idx < cnt; idx += blockDim.x) {
      const int i = k + 1 + idx / w, c = idx % w;
      const dfl f = df_mul(upk(G[i * RS + k]), dk);
      G[c * RS + i + 1] = pk(df_sub(upk(G[c * RS + i + 1]), df_mul(f, upk(G[c * RS + k + 1]))));
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < RR; idx += blockDim.x) {
    const int i = idx / R, c = idx % R;
    const dfl val = c <= i ? df_mul(upk(G[c * RS + i + 1]), upk(dinv[i])) : dfl{0.f, 0.f};
    tp[b.lih + idx] = val.hi;
    tp[b.lil + idx] = val.lo;
  }
}

// Row solves through W = L^-1 (u = b W^T, a = u W) in double-float; b = rhs
// + A_old Z (float; the sum of two floats is exact as a double-float).  The
// new factor keeps its high and low words (compute copy and alo) and its
// float64 value; dA = A_new - A_old (ALS) or A_new - A_p (PP) in
// double-float, its compute copy in float; row norms in float.
constexpr size_t bsolve_df_smem() {
  return (size_t)kBR * (kBR + 1) * (sizeof(float2) + sizeof(float)) +
         2 * (size_t)kSolveTR * (kBR + 1) * sizeof(float2);
}

__global__ void __launch_bounds__(256) bsolve_df_kernel(BParams P, int stage, int n, float* __restrict__ tp,
                                                        double* __restrict__ dp) {
  const BI& b = P.bi[blockIdx.y];
  const BC c = P.ctl[blockIdx.y];
  if (!ne_active(stage, c)) return;
  const int R = b.R, s = b.s[n], RS = kBR + 1;
  const bool failed = (c.status >> n) & 1;
  if (failed) return;                            // the mode keeps its factor and dA
  const bool dense = (c.status >> (16 + n)) & 1;   // W from Gamma^dagger: no zero triangle
  const bool als = ne_als(stage, c);
  const bool v = ne_pp(stage, c) && P.use_V;
  extern __shared__ __align__(16) unsigned char bs_raw[];
  float2* Ws = reinterpret_cast<float2*>(bs_raw);
  float2* bt = Ws + kBR * RS;
  float2* ut = bt + kSolveTR * RS;
  float* Zs = reinterpret_cast<float*>(ut + kSolveTR * RS);
  for (int idx = threadIdx.x; idx < R * R; idx += blockDim.x) {
    const int o = (idx / R) * RS + idx % R;
    Ws[o] = make_float2(tp[b.lih + idx], tp[b.lil + idx]);
    if (v) Zs[o] = tp[b.zf + idx];
  }
  const float* rhs = tp + (als && n == 2 ? b.mr : b.rhs);
  float* Ah = tp + b.ac[n];
  float* Al = tp + b.alo[n];
  const float* Rh = tp + (als ? b.ac[n] : b.aph[n]);
  const float* Rl = tp + (als ? b.alo[n] : b.apl[n]);
  float* dAc = tp + b.dac[n];
  float* rhs2 = tp + b.rhs2;
  double* A = dp + b.a[n];
  double* rn = dp + b.rn;
  const int t = threadIdx.x >> 4, l = threadIdx.x & 15;
  const int nq = (R + 15) >> 4;
  for (int y0 = blockIdx.x * kSolveTR; y0 < s; y0 += gridDim.x * kSolveTR) {
    const int y = y0 + t;
    const bool on = y < s;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int r = l + 16 * q;
      if (q >= nq || r >= R) continue;
      const float bv = on ? rhs[(int64_t)y * R + r] : 0.f;
      dfl bd{bv, 0.f};
      if (v && on) {
        float acc = 0.f;
        const float* ar = Ah + (int64_t)y * R;
        for (int k = 0; k < R; k++) acc = fmaf(ar[k], Zs[k * RS + r], acc);
        bd = two_sum(bv, acc);
        if (n == 2) rhs2[(int64_t)y * R + r] = bd.hi;
      }
      bt[t * RS + r] = pk(bd);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; q++) {
      if (q >= nq) break;
      const int j = l + 16 * q;
      const int kend = dense ? R - 1 : min(16 * q + 15, R - 1);
      dfl u{0.f, 0.f};
      for (int k = 0; k <= kend; k++)
        if (dense || k <= j) u = df_add(u, df_mul(upk(bt[t * RS + k]), upk(Ws[j * RS + k])));
      if (j < R) ut[t * RS + j] = pk(u);
    }
    __syncthreads();
    float nd = 0.f, na = 0.f;
#pragma unroll
    for (int q = 0; q < 4; q++) {
      if (q >= nq) break;
      const int r = l + 16 * q;
      dfl a{0.f, 0.f};
      for (int j = dense ? 0 : 16 * q; j < R; j++)
        if (dense || j >= r) a = df_add(a, df_mul(upk(ut[t * RS + j]), upk(Ws[j * RS + r])));
      if (r >= R || !on) continue;
      const int64_t o = (int64_t)y * R + r;
      const dfl d = df_sub(a, dfl{Rh[o], Rl[o]});   // reads A_old before it is replaced
      Ah[o] = a.hi;
      Al[o] = a.lo;
      A[o] = (double)a.hi + (double)a.lo;
      dAc[o] = d.hi;
      nd = fmaf(d.hi, d.hi, nd);
      na = fmaf(a.hi, a.hi, na);
    }
#pragma unroll
    for (int off = 8; off > 0; off >>= 1) {
      nd += __shfl_xor_sync(0xffffffffu, nd, off);
      na += __shfl_xor_sync(0xffffffffu, na, off);
    }
    if (l == 0 && on) {
      rn[2 * y] = nd;
      rn[2 * y + 1] = na;
    }
  }
}

// Grams of mode n in double-float: S^(n) = A^T A from the factor's high and
// low words (32 x 32 blocks as the float64 kernel, row order), written as
// double-float and as float64; W^(n) = A^T dA in float; CTA 0 sums the row
// norms.
__global__ void __launch_bounds__(256) bgram_df_kernel(BParams P, int stage, int n, float* __restrict__ tp,
                                                       double* __restrict__ dp) {
  const BI& b = P.bi[blockIdx.y];
  const BC c = P.ctl[blockIdx.y];
  if (!ne_active(stage, c)) return;
  const int R = b.R, s = b.s[n];
  const int nb = (R + 31) >> 5;
  const int nS = nb * (nb + 1) / 2;
  const int nW = ne_pp(stage, c) ? nb * nb : 0;
  const int blk = blockIdx.x;
  const int ti = threadIdx.x >> 4, tj = threadIdx.x & 15;
  __shared__ float2 xs[32 * 33], ys[32 * 33];
  if (blk < nS) {
    const int bi = blk >= 1, bj = blk == 2;
    const int i0 = 32 * bi, j0 = 32 * bj;
    const float* Ah = tp + b.ac[n];
    const float* Al = tp + b.alo[n];
    dfl acc[2][2];
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
      for (int e = 0; e < 2; e++) acc[a][e] = dfl{0.f, 0.f};
    for (int y0 = 0; y0 < s; y0 += 32) {
      __syncthreads();
      for (int idx = threadIdx.x; idx < 32 * 32; idx += blockDim.x) {
        const int yy = idx >> 5, cc = idx & 31, y = y0 + yy;
        const bool okx = y < s && i0 + cc < R, oky = y < s && j0 + cc < R;
        xs[yy * 33 + cc] = okx ? make_float2(Ah[(int64_t)y * R + i0 + cc], Al[(int64_t)y * R + i0 + cc])
                               : make_float2(0.f, 0.f);
        ys[yy * 33 + cc] = oky ? make_float2(Ah[(int64_t)y * R + j0 + cc], Al[(int64_t)y * R + j0 + cc])
                               : make_float2(0.f, 0.f);
      }
      __syncthreads();
      const int ye = min(32, s - y0);
      for (int yy = 0; yy < ye; yy++) {
        const dfl x0 = upk(xs[yy * 33 + ti]), x1 = upk(xs[yy * 33 + ti + 16]);
        const dfl z0 = upk(ys[yy * 33 + tj]), z1 = upk(ys[yy * 33 + tj + 16]);
        acc[0][0] = df_add(acc[0][0], df_mul(x0, z0));
        acc[0][1] = df_add(acc[0][1], df_mul(x0, z1));
        acc[1][0] = df_add(acc[1][0], df_mul(x1, z0));
        acc[1][1] = df_add(acc[1][1], df_mul(x1, z1));
      }
    }
    float* shn = tp + b.shi + (int64_t)n * R * R;
    float* sln = tp + b.slo + (int64_t)n * R * R;
    double* S = dp + b.S + (int64_t)n * R * R;
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
      for (int e = 0; e < 2; e++) {
        const int i = i0 + ti + 16 * a, j = j0 + tj + 16 * e;
        if (i < R && j < R) {
          const dfl v = acc[a][e];
          const double vd = (double)v.hi + (double)v.lo;
          shn[i * R + j] = v.hi;
          sln[i * R + j] = v.lo;
          S[i * R + j] = vd;
          if (bi != bj) {
            shn[j * R + i] = v.hi;
            sln[j * R + i] = v.lo;
            S[j * R + i] = vd;
          }
        }
      }
  } else if (blk < nS + nW) {
    const int f = blk - nS, i0 = 32 * (f / nb), j0 = 32 * (f % nb);
    float acc[2][2];
    float* gx = reinterpret_cast<float*>(xs);
    gram_block<float>(tp + b.ac[n], tp + b.dac[n], s, R, i0, j0, gx, gx + 32 * 33, acc);
    float* Wn = tp + b.wg + (int64_t)n * R * R;
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
      for (int e = 0; e < 2; e++) {
        const int i = i0 + ti + 16 * a, j = j0 + tj + 16 * e;
        if (i < R && j < R) Wn[i * R + j] = acc[a][e];
      }
  }
  if (blk != 0) return;
  __shared__ double rd[256], ra[256];
  double x = 0.0, z = 0.0;
  if (stage == NE_INIT) {
    const double* A = dp + b.a[n];
    for (int64_t e = threadIdx.x; e < (int64_t)s * R; e += blockDim.x) z = fma(A[e], A[e], z);
    x = z;
  } else {
    for (int y = threadIdx.x; y < s; y += blockDim.x) {
      x += dp[b.rn + 2 * y];
      z += dp[b.rn + 2 * y + 1];
    }
  }
  rd[threadIdx.x] = x;
  ra[threadIdx.x] = z;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) {
      rd[threadIdx.x] += rd[threadIdx.x + st];
      ra[threadIdx.x] += ra[threadIdx.x + st];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    dp[b.sc + 8 + 2 * n] = rd[0];
    dp[b.sc + 9 + 2 * n] = ra[0];
  }
}

// ---------------------------------------------------------------- PP sweep, fitness, controller
// Eq. 3 first-order terms of mode n: rhs[y][r] = M_p^(n)[y][r] +
// sum_{i != n} sum_x M_p^(i,n)(x, y, r) dA^(i)[x][r] with the operators
// M_p^(0,1)[x0][x1][r], M_p^(0,2)[x0][x2][r], M_p^(1,2)[x1][x2][r].
template <typename T>
__global__ void __launch_bounds__(256, 4) bppcorr_kernel(BParams P, int n, T* __restrict__ tp) {
  const BI& b = P.bi[blockIdx.y];   // fields read once, indexed by mode
  if (!runs_pp(P.ctl[blockIdx.y])) return;
  const int R = b.R;
  const int s0 = b.s[0], s1 = b.s[1], s2 = b.s[2];
  // two terms: operator base for row y = base + y * ystride, x stride, extent, dA
  int64_t base0, base1;
  int ys0, ys1, xs0, xs1, sx0, sx1;
  const T *d0, *d1;
  if (n == 0) {
    base0 = b.op01; ys0 = s1 * R; xs0 = R; sx0 = s1; d0 = tp + b.dac[1];
    base1 = b.op02; ys1 = s2 * R; xs1 = R; sx1 = s2; d1 = tp + b.dac[2];
  } else if (n == 1) {
    base0 = b.op01; ys0 = R; xs0 = s1 * R; sx0 = s0; d0 = tp + b.dac[0];
    base1 = b.op12; ys1 = s2 * R; xs1 = R; sx1 = s2; d1 = tp + b.dac[2];
  } else {
    base0 = b.op02; ys0 = R; xs0 = s2 * R; sx0 = s0; d0 = tp + b.dac[0];
    base1 = b.op12; ys1 = R; xs1 = s2 * R; sx1 = s1; d1 = tp + b.dac[1];
  }
  // 32 consecutive outputs per CTA pass; the 8 warps split each sum over x
  // (x = warp, warp + 8, ...), the two terms in separate accumulators so
  // that both operators' loads are in flight together, and the partials
  // are added in warp order
  const int tot = b.s[n] * R;
  const int o = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int sxm = min(sx0, sx1);
  const T* mp = tp + b.mp[n];
  T* rhs = tp + b.rhs;
  __shared__ T part[8][33];
  for (int c0 = blockIdx.x * 32; c0 < tot; c0 += gridDim.x * 32) {
    const int i = c0 + o;
    T acc0 = T(0), acc1 = T(0);
    if (i < tot) {
      const int y = i / R, r = i - y * R;
      // pointers stepped by 8 rows of x
      const T* p0 = tp + base0 + (int64_t)y * ys0 + r + (int64_t)g * xs0;
      const T* p1 = tp + base1 + (int64_t)y * ys1 + r + (int64_t)g * xs1;
      const T* q0 = d0 + r + g * R;
      const T* q1 = d1 + r + g * R;
      const int64_t st0 = 8 * (int64_t)xs0, st1 = 8 * (int64_t)xs1;
      const int stq = 8 * R;
      int x = g;
#pragma unroll 4
      for (; x < sxm; x += 8) {
        acc0 = fma(*p0, *q0, acc0);
        acc1 = fma(*p1, *q1, acc1);
        p0 += st0; p1 += st1; q0 += stq; q1 += stq;
      }
      for (int x0 = x; x0 < sx0; x0 += 8, p0 += st0, q0 += stq) acc0 = fma(*p0, *q0, acc0);
      for (int x1 = x; x1 < sx1; x1 += 8, p1 += st1, q1 += stq) acc1 = fma(*p1, *q1, acc1);
    }
    part[g][o] = acc0 + acc1;
    __syncthreads();
    if (g == 0 && i < tot) {
      T sum = mp[i];
#pragma unroll
      for (int k = 0; k < 8; k++) sum += part[k][o];
      rhs[i] = sum;
    }
    __syncthreads();
  }
}

// The PP initialisation of Algorithm 3 after the operator build: A_p <- A,
// dA <- 0 (float64 and compute copies), W <- 0, ||dA||^2 <- 0.
template <typename T>
__global__ void bprep_kernel(BParams P, T* __restrict__ tp, double* __restrict__ dp) {
  const BI b = P.bi[blockIdx.y];
  if (!runs_init(P.ctl[blockIdx.y])) return;
  const int R = b.R;
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, st = (int64_t)gridDim.x * blockDim.x;
  for (int n = 0; n < 3; n++)
    for (int64_t i = g; i < (int64_t)b.s[n] * R; i += st) {
      dp[b.ap[n] + i] = dp[b.a[n] + i];
      dp[b.da[n] + i] = 0.0;
      tp[b.dac[n] + i] = T(0);
      tp[b.aph[n] + i] = tp[b.ac[n] + i];
      tp[b.apl[n] + i] = tp[b.alo[n] + i];
    }
  for (int64_t i = g; i < 3 * (int64_t)R * R; i += st) {
    dp[b.W + i] = 0.0;
    tp[b.wg + i] = T(0);
  }
  if (g < 3) dp[b.sc + 8 + 2 * g] = 0.0;
}

// Fitness (Sec. 5): 1 - sqrt(||X||^2 - 2 <X, [[A]]> + ||[[A]]||^2) / ||X||, the
// inner product from the last mode's right-hand side and new factor: exact
// after ALS sweeps and in the exact pass (M^(2) = X_(01)^T (A^(0) (.) A^(1))),
// the estimate from M~^(2) after PP sweeps (with the second-order terms when
// they are on).  One CTA per instance, float64 sums.
template <typename T>
__global__ void __launch_bounds__(256) bfit_kernel(BParams P, T* __restrict__ tp, double* __restrict__ dp) {
  const BI b = P.bi[blockIdx.y];
  const BC c = P.ctl[blockIdx.y];
  if (c.ran == K_DONE) return;
  const int R = b.R;
  const T* rhs = tp + (runs_right(c) ? b.mr : (P.use_V ? b.rhs2 : b.rhs));
  const double* A2 = dp + b.a[2];
  const double* S = dp + b.S;
  double inner = 0.0, model = 0.0;
  for (int64_t i = threadIdx.x; i < (int64_t)b.s[2] * R; i += blockDim.x)
    inner = fma((double)rhs[i], A2[i], inner);
  for (int i = threadIdx.x; i < R * R; i += blockDim.x) model += S[i] * S[R * R + i] * S[2 * R * R + i];
  __shared__ double ri[256], rm[256];
  ri[threadIdx.x] = inner;
  rm[threadIdx.x] = model;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) {
      ri[threadIdx.x] += ri[threadIdx.x + st];
      rm[threadIdx.x] += rm[threadIdx.x + st];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double nx2 = dp[b.sc + 3];
    const double res2 = nx2 - 2.0 * ri[0] + rm[0];
    dp[b.sc + 0] = 1.0 - sqrt(fmax(res2, 0.0)) / sqrt(nx2);
    dp[b.sc + 1] = ri[0];
    dp[b.sc + 2] = rm[0];
  }
}

__device__ bool b_all_small(const BParams& P, const BI& b, const double* dp) {
  if (!(P.eps > 0.0)) return false;
  for (int n = 0; n < 3; n++)
    if (!(sqrt(dp[b.sc + 8 + 2 * n]) < P.eps * sqrt(dp[b.sc + 9 + 2 * n]))) return false;
  return true;
}

// Algorithm 3's decision per instance after a sweep (one thread each): the
// sweep is recorded (kind, the fitness it reports), then the next kind is
// taken as the host loop of cpals_run does -- after an ALS sweep a PP
// initialisation iff every ||dA^(i)|| < eps ||A^(i)||; inside a PP run
// another PP sweep iff that still holds and, with a stopping tolerance, the
// last PP sweep of the run (from its second on) raised the estimate by at
// least tol; else an ALS sweep.  A non-finite value or a failed
// factorisation ends the instance; so does its sweep budget.
// first != 0: the decision before the first sweep (dA = A).
__global__ void bdecide_kernel(BParams P, int n_inst, int first, double* __restrict__ dp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_inst) return;
  BC& c = P.ctl[i];
  const BI b = P.bi[i];
  if (first) {
    c.t = 0;
    c.in_run = 0;
    c.status = 0;
    c.f_last = c.f_prev = -1e300;
    c.ran = c.next = P.max_sweeps > 0 ? (b_all_small(P, b, dp) ? K_INIT : K_ALS) : K_DONE;
    return;
  }
  if (c.ran == K_DONE || c.ran == K_EXACT) return;
  const double f = dp[b.sc + 0];
  const int t = c.t;
  P.ftrace[(int64_t)i * P.max_sweeps + t] = f;
  P.ktrace[(int64_t)i * P.max_sweeps + t] = c.ran;
  c.t = t + 1;
  c.f_prev = c.f_last;
  c.f_last = f;
  c.in_run = c.ran == K_ALS ? 0 : (c.ran == K_INIT ? 1 : c.in_run + 1);
  bool finite = isfinite(f);
  for (int n = 0; n < 3; n++) finite = finite && isfinite(dp[b.sc + 8 + 2 * n]) && isfinite(dp[b.sc + 9 + 2 * n]);
  if (!finite) c.status |= 1 << 8;
  if ((c.status & 0xffff) || c.t >= P.max_sweeps) {   // bits 16 + n: Gamma^dagger used
    c.ran = c.next = K_DONE;
    return;
  }
  const bool small = b_all_small(P, b, dp);
  const bool gain = !(P.tol > 0.0) || c.in_run < 2 || c.f_last - c.f_prev >= P.tol;
  c.next = c.ran != K_ALS ? ((small && gain) ? K_PP : K_ALS) : (small ? K_INIT : K_ALS);
  c.ran = c.next;
}

// The exact pass after the last sweep: every instance that ran takes the
// exact fitness of its final factors (stage flag K_EXACT), then ends.
__global__ void bexact_kernel(BParams P, int n_inst, int begin) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_inst) return;
  BC& c = P.ctl[i];
  if (begin) c.ran = c.t > 0 ? K_EXACT : K_DONE;
  else c.ran = K_DONE;
}

// Compute copies and dA of the initial factors: Ac = dAc = A, dA = A, W = 0.
template <typename T>
__global__ void binit_kernel(BParams P, T* __restrict__ tp, double* __restrict__ dp) {
  const BI b = P.bi[blockIdx.y];
  const int R = b.R;
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, st = (int64_t)gridDim.x * blockDim.x;
  for (int n = 0; n < 3; n++)
    for (int64_t i = g; i < (int64_t)b.s[n] * R; i += st) {
      const double a = dp[b.a[n] + i];
      dp[b.da[n] + i] = a;
      tp[b.ac[n] + i] = (T)a;
      tp[b.dac[n] + i] = (T)a;
      if constexpr (sizeof(T) == 4) tp[b.alo[n] + i] = (T)(a - (double)(T)a);
    }
  for (int64_t i = g; i < 3 * (int64_t)R * R; i += st) {
    dp[b.W + i] = 0.0;
    tp[b.wg + i] = T(0);
  }
}

// ||X||^2 of instance i in float64 (one CTA, fixed order).
template <typename T>
__global__ void __launch_bounds__(256) bnormx_kernel(const T* __restrict__ X, int64_t n, double* __restrict__ out) {
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc = fma((double)X[i], (double)X[i], acc);
  __shared__ double r[256];
  r[threadIdx.x] = acc;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) r[threadIdx.x] += r[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = r[0];
}

template <typename TS, typename TD>
__global__ void bconvert_kernel(const TS* __restrict__ s, TD* __restrict__ d, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    d[i] = (TD)s[i];
}

}  // namespace

// ====================================================================== host side
struct cpals_batch {
  int n = 0, prec = 0;
  size_t esz = 4;
  std::vector<BI> bi;
  BI* d_bi = nullptr;
  BC* d_ctl = nullptr;
  void* tp = nullptr;
  double* dp = nullptr;
  int64_t tp_elems = 0, dp_elems = 0;
  std::vector<char> have_x, have_a;
  cudaStream_t stream = nullptr;
  double* d_ftrace = nullptr;
  int* d_ktrace = nullptr;
  int64_t trace_cap = 0;
  // grid extents (largest over the instances)
  int64_t u_l = 1, u_r = 1, u_12 = 1, u_02 = 1, smax = 1, el_max = 1;
  int64_t launches_sweep = 0, launches_run = 0;
  // tile configuration of the M^(L) and mode-2 contraction stages (autotuner)
  int tile[kTuneStages] = {0, 0, 0, 0};
  float tile_ms[kTuneStages][kTileCfgs] = {{-1.f, -1.f, -1.f}, {-1.f, -1.f, -1.f}, {-1.f, -1.f, -1.f},
                                           {-1.f, -1.f, -1.f}};
  bool tuned = false, tile_from_cache = false;
  std::string err;
  cpals_status fail(cpals_status st, const std::string& m) {
    err = m;
    return st;
  }
  cpals_status cuda_fail(const char* what, cudaError_t e) {
    err = std::string(what) + ": " + cudaGetErrorString(e);
    return CPALS_E_CUDA;
  }
};

#define CKS_B(expr)                    \
  do {                                 \
    cpals_status s_ = (expr);          \
    if (s_ != CPALS_OK) return s_;     \
  } while (0)

#define BCK(call)                                           \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return b->cuda_fail(#call, e_);  \
  } while (0)

namespace {

int el_grid(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(n, kBT), 64)); }
constexpr int64_t kGemmCtas = 32;   // CTAs per instance of a contraction stage (they loop over its units)

// One contraction stage with tile configuration cfg (0: 64-row tiles,
// 1: 128-row tiles).
template <typename T>
void launch_gemm(const cpals_batch* b, const BParams& P, int stage, int64_t units, int cfg) {
  const dim3 g((unsigned)std::min<int64_t>(units, kGemmCtas), (unsigned)b->n);
  T* tp = static_cast<T*>(b->tp);
  if (cfg == 1) bgemm_kernel<T, 128, 8><<<g, kBT, 0, b->stream>>>(P, stage, tp);
  else if (cfg == 2) bgemm_kernel<T, 32, 2><<<g, kBT, 0, b->stream>>>(P, stage, tp);
  else bgemm_kernel<T, 64, 4><<<g, kBT, 0, b->stream>>>(P, stage, tp);
}

// Tile autotuner: for each of the four contraction stages (M^(L), the mode-2
// right-hand side, M_p^(1,2), M_p^(0,2)) each tile configuration is timed on
// the batch itself with every instance taking part (CUDA events, one
// warm-up and three timed launches) and the fastest kept; results are cached per batch signature (sizes,
// ranks, precision) for the life of the process, so later batches of the
// same shapes reuse them without timing.
std::mutex g_tune_mutex;
std::map<uint64_t, std::array<int, kTuneStages>> g_tune_cache;

uint64_t batch_signature(const cpals_batch* b) {
  uint64_t h = 1469598103934665603ull ^ (uint64_t)b->esz;
  auto mix = [&](uint64_t v) { h = (h ^ v) * 1099511628211ull; };
  for (const BI& q : b->bi) {
    mix((uint64_t)q.s[0]);
    mix((uint64_t)q.s[1]);
    mix((uint64_t)q.s[2]);
    mix((uint64_t)q.R);
  }
  return h;
}

template <typename T>
cpals_status autotune(cpals_batch* b, const BParams& P) {
  if (b->tuned) return CPALS_OK;
  const uint64_t key = batch_signature(b);
  {
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      for (int st = 0; st < kTuneStages; st++) b->tile[st] = it->second[st];
      b->tuned = true;
      b->tile_from_cache = true;
      return CPALS_OK;
    }
  }
  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0));
  BCK(cudaEventCreate(&e1));
  // every instance takes part in the timed launches (their outputs are
  // scratch until the sweeps write them)
  BParams Pf = P;
  Pf.force = 1;
  const int64_t units[kTuneStages] = {b->u_l, b->u_r, b->u_12, b->u_02};
  for (int st = 0; st < kTuneStages; st++) {
    float best = 0.f;
    for (int cfg = 0; cfg < kTileCfgs; cfg++) {
      launch_gemm<T>(b, Pf, st, units[st], cfg);
      cudaEventRecord(e0, b->stream);
      for (int rep = 0; rep < 3; rep++) launch_gemm<T>(b, Pf, st, units[st], cfg);
      cudaEventRecord(e1, b->stream);
      cudaError_t e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return b->cuda_fail("autotune", e);
      }
      b->tile_ms[st][cfg] = ms / 3.f;
      if (cfg == 0 || ms < best) {
        best = ms;
        b->tile[st] = cfg;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->tuned = true;
  b->tile_from_cache = false;
  std::lock_guard<std::mutex> lk(g_tune_mutex);
  g_tune_cache[key] = {b->tile[0], b->tile[1], b->tile[2], b->tile[3]};
  return CPALS_OK;
}

// Launch every stage of one sweep of the whole batch (captured into a graph).
template <typename T>
int64_t sweep_launches(cpals_batch* b, const BParams& P) {
  T* tp = static_cast<T*>(b->tp);
  double* dp = b->dp;
  cudaStream_t s = b->stream;
  const unsigned N = (unsigned)b->n;
  int64_t k = 0;
  auto gemm = [&](int stage, int64_t units) {
    const int cfg = b->tile[stage];
    launch_gemm<T>(b, P, stage, units, cfg);
    k++;
  };
  const dim3 gsolve((unsigned)std::min<int64_t>(kSolveCtas, cdiv(b->smax, kSolveTR)), N);
  const dim3 gel((unsigned)el_grid(b->el_max), N);
  auto mode = [&](int stage, int n) {
    if constexpr (sizeof(T) == 4) {
      bchol_df_kernel<<<dim3(1, N), 256, 0, s>>>(P, stage, n, tp, dp);
      bsolve_df_kernel<<<gsolve, 256, bsolve_df_smem(), s>>>(P, stage, n, tp, dp);
      bgram_df_kernel<<<dim3(kGramCtas, N), 256, 0, s>>>(P, stage, n, tp, dp);
    } else {
      bchol_kernel<<<dim3(1, N), 128, 0, s>>>(P, stage, n, dp);
      bsolve_kernel<T><<<gsolve, 256, bsolve_smem<T>(), s>>>(P, stage, n, tp, dp);
      bgram_kernel<T><<<dim3(kGramCtas, N), 256, 0, s>>>(P, stage, n, tp, dp);
    }
    k += 3;
  };
  // M^(L) (ALS, Sec. 2.5), which doubles as M_p^(0,1) for the instances
  // that build operators; the rest of the operator build (Sec. 3.2.3) and
  // the PP initialisation of Algorithm 3
  gemm(CT_L, b->u_l);
  gemm(CT_12, b->u_12);
  gemm(CT_02, b->u_02);
  bttv_kernel<T><<<dim3(gel.x, N, 3), kBT, 0, s>>>(P, TT_MP, tp);
  bprep_kernel<T><<<gel, kBT, 0, s>>>(P, tp, dp);
  k += 2;
  // modes 0, 1, 2 (Gauss-Seidel): each instance forms its right-hand side
  // (ALS: the dimension tree; PP: Eq. 3), then one factorisation, solve and
  // Gram stage serves both sweep kinds
  bttv_kernel<T><<<gel, kBT, 0, s>>>(P, TT_ALS0, tp);
  bppcorr_kernel<T><<<gel, kBT, 0, s>>>(P, 0, tp);
  k += 2;
  mode(NE_SWEEP, 0);
  bttv_kernel<T><<<gel, kBT, 0, s>>>(P, TT_ALS1, tp);
  bppcorr_kernel<T><<<gel, kBT, 0, s>>>(P, 1, tp);
  k += 2;
  mode(NE_SWEEP, 1);
  bkrp_kernel<T><<<gel, kBT, 0, s>>>(P, tp);
  gemm(CT_R, b->u_r);
  breduce_kernel<T><<<gel, kBT, 0, s>>>(P, tp);
  bppcorr_kernel<T><<<gel, kBT, 0, s>>>(P, 2, tp);
  k += 3;
  mode(NE_SWEEP, 2);
  bfit_kernel<T><<<dim3(1, N), 256, 0, s>>>(P, tp, dp);
  bdecide_kernel<<<(unsigned)cdiv(b->n, 128), 128, 0, s>>>(P, b->n, 0, dp);
  return k + 2;
}

// The exact fitness of every instance's final factors.
template <typename T>
int64_t exact_launches(cpals_batch* b, const BParams& P) {
  T* tp = static_cast<T*>(b->tp);
  cudaStream_t s = b->stream;
  const unsigned N = (unsigned)b->n;
  const dim3 gel((unsigned)el_grid(b->el_max), N);
  bexact_kernel<<<(unsigned)cdiv(b->n, 128), 128, 0, s>>>(P, b->n, 1);
  bkrp_kernel<T><<<gel, kBT, 0, s>>>(P, tp);
  launch_gemm<T>(b, P, CT_R, b->u_r, b->tile[CT_R]);
  breduce_kernel<T><<<gel, kBT, 0, s>>>(P, tp);
  bfit_kernel<T><<<dim3(1, N), 256, 0, s>>>(P, tp, b->dp);
  bexact_kernel<<<(unsigned)cdiv(b->n, 128), 128, 0, s>>>(P, b->n, 0);
  return 6;
}

template <typename T>
cpals_status run_impl(cpals_batch* b, int max_sweeps, double eps, int use_V, double tol) {
  T* tp = static_cast<T*>(b->tp);
  double* dp = b->dp;
  cudaStream_t s = b->stream;
  const unsigned N = (unsigned)b->n;
  BParams P{};                       // force = 0: stages follow each instance's sweep kind
  P.bi = b->d_bi;
  P.ctl = b->d_ctl;
  P.eps = eps;
  P.tol = tol;
  P.use_V = use_V;
  P.max_sweeps = max_sweeps;
  P.ftrace = b->d_ftrace;
  P.ktrace = b->d_ktrace;
  // Algorithm 3's start: dA <- A, S <- A^T A, the first decision
  BCK(cudaMemsetAsync(b->d_ctl, 0, sizeof(BC) * b->n, s));
  binit_kernel<T><<<dim3((unsigned)el_grid(b->el_max), N), kBT, 0, s>>>(P, tp, dp);
  for (int n = 0; n < 3; n++) {
    if constexpr (sizeof(T) == 4) bgram_df_kernel<<<dim3(kGramCtas, N), 256, 0, s>>>(P, NE_INIT, n, tp, dp);
    else bgram_kernel<T><<<dim3(kGramCtas, N), 256, 0, s>>>(P, NE_INIT, n, tp, dp);
  }
  bdecide_kernel<<<(unsigned)cdiv(b->n, 128), 128, 0, s>>>(P, b->n, 1, dp);
  BCK(cudaGetLastError());
  CKS_B(autotune<T>(b, P));
  int64_t launches = 5;
  // one captured graph is one sweep of every instance
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr, exx = nullptr;
  BCK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  const int64_t per = sweep_launches<T>(b, P);
  cudaError_t e = cudaStreamEndCapture(s, &g);
  if (e != cudaSuccess) return b->cuda_fail("capture (batch sweep)", e);
  e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return b->cuda_fail("instantiate (batch sweep)", e);
  BCK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  const int64_t nex = exact_launches<T>(b, P);
  e = cudaStreamEndCapture(s, &g);
  if (e == cudaSuccess) {
    e = cudaGraphInstantiate(&exx, g, 0);
    cudaGraphDestroy(g);
  }
  if (e != cudaSuccess) {
    cudaGraphExecDestroy(ex);
    return b->cuda_fail("capture (batch exact fitness)", e);
  }
  for (int t = 0; t < max_sweeps && e == cudaSuccess; t++) e = cudaGraphLaunch(ex, s);
  if (e == cudaSuccess) e = cudaGraphLaunch(exx, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaGraphExecDestroy(ex);
  cudaGraphExecDestroy(exx);
  if (e != cudaSuccess) return b->cuda_fail("batch run", e);
  b->launches_sweep = per;
  b->launches_run = launches + per * max_sweeps + nex;
  return CPALS_OK;
}

}  // namespace

extern "C" {

cpals_status cpals_batch_create(int n, const int64_t* dims, const int* ranks, int precision,
                                cpals_batch** out) {
  if (!out) return CPALS_E_INVALID;
  *out = nullptr;
  if (n < 1 || n > 65535 || !dims || !ranks) return CPALS_E_INVALID;
  if (precision != CPALS_FP64 && precision != CPALS_FP32) return CPALS_E_UNSUPPORTED;
  for (int i = 0; i < n; i++) {
    if (ranks[i] < 1 || ranks[i] > kBR) return CPALS_E_INVALID;
    for (int k = 0; k < 3; k++)
      if (dims[3 * i + k] < 1 || dims[3 * i + k] > 4096) return CPALS_E_INVALID;
  }
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    cudaGetLastError();
    return CPALS_E_CUDA;
  }
  if (!(prop.major == 10 && prop.minor == 3)) return CPALS_E_UNSUPPORTED;
  if (cudaFuncSetAttribute(bsolve_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)bsolve_smem<double>()) != cudaSuccess ||
      cudaFuncSetAttribute(bsolve_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)bsolve_df_smem()) != cudaSuccess) {
    cudaGetLastError();
    return CPALS_E_CUDA;
  }
  cpals_batch* b = new cpals_batch();
  b->n = n;
  b->prec = precision;
  b->esz = precision == CPALS_FP64 ? 8 : 4;
  b->bi.resize(n);
  b->have_x.assign(n, 0);
  b->have_a.assign(n, 0);
  int64_t to = 0, d = 0;
  for (int i = 0; i < n; i++) {
    BI& q = b->bi[i];
    memset(&q, 0, sizeof(q));
    const int64_t s0 = dims[3 * i], s1 = dims[3 * i + 1], s2 = dims[3 * i + 2];
    const int R = ranks[i];
    q.s[0] = (int)s0;
    q.s[1] = (int)s1;
    q.s[2] = (int)s2;
    q.R = R;
    const int64_t K = s0 * s1;
    q.splits = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(K, 1024), 64));
    const int64_t sm = std::max(s0, std::max(s1, s2));
    auto t = [&](int64_t e) { const int64_t o = to; to += (e + 1) / 2 * 2; return o; };
    q.x = t(s0 * s1 * s2);
    for (int k = 0; k < 3; k++) q.ac[k] = t(dims[3 * i + k] * R);
    for (int k = 0; k < 3; k++) q.dac[k] = t(dims[3 * i + k] * R);
    q.ml = t(K * R);
    q.mr = t(s2 * R);
    q.krp = t(K * R);
    q.rhs = t(sm * R);
    q.rhs2 = t(sm * R);
    q.part = t((int64_t)q.splits * s2 * R);
    q.op01 = t(s0 * s1 * R);
    q.op02 = t(s0 * s2 * R);
    q.op12 = t(s1 * s2 * R);
    for (int k = 0; k < 3; k++) q.mp[k] = t(dims[3 * i + k] * R);
    for (int k = 0; k < 3; k++) q.alo[k] = t(dims[3 * i + k] * R);
    for (int k = 0; k < 3; k++) q.aph[k] = t(dims[3 * i + k] * R);
    for (int k = 0; k < 3; k++) q.apl[k] = t(dims[3 * i + k] * R);
    q.shi = t(3 * (int64_t)R * R);
    q.slo = t(3 * (int64_t)R * R);
    q.lih = t((int64_t)R * R);
    q.lil = t((int64_t)R * R);
    q.wg = t(3 * (int64_t)R * R);
    q.zf = t((int64_t)R * R);
    auto dd = [&](int64_t e) { const int64_t o = d; d += e; return o; };
    for (int k = 0; k < 3; k++) q.a[k] = dd(dims[3 * i + k] * R);
    for (int k = 0; k < 3; k++) q.ap[k] = dd(dims[3 * i + k] * R);
    for (int k = 0; k < 3; k++) q.da[k] = dd(dims[3 * i + k] * R);
    q.S = dd(3 * (int64_t)R * R);
    q.W = dd(3 * (int64_t)R * R);
    q.L = dd((int64_t)R * R);
    q.Z = dd((int64_t)R * R);
    q.rn = dd(2 * sm);
    q.sc = dd(16);
    b->u_l = std::max(b->u_l, cdiv(K, 64));
    b->u_r = std::max(b->u_r, cdiv(s2, 64) * q.splits);
    b->u_12 = std::max(b->u_12, cdiv(s1 * s2, 64));
    b->u_02 = std::max(b->u_02, cdiv(s2, 64) * s0);
    b->smax = std::max(b->smax, sm);
    b->el_max = std::max(b->el_max, K * R);
  }
  b->tp_elems = to;
  b->dp_elems = d;
  auto bail = [&](cpals_status st) {
    cpals_batch_destroy(b);
    return st;
  };
  if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(CPALS_E_CUDA);
  if (cudaMalloc(&b->tp, (size_t)to * b->esz) != cudaSuccess ||
      cudaMalloc((void**)&b->dp, (size_t)d * 8) != cudaSuccess ||
      cudaMalloc((void**)&b->d_bi, sizeof(BI) * n) != cudaSuccess ||
      cudaMalloc((void**)&b->d_ctl, sizeof(BC) * n) != cudaSuccess) {
    cudaGetLastError();
    return bail(CPALS_E_OOM);
  }
  if (cudaMemcpy(b->d_bi, b->bi.data(), sizeof(BI) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(b->dp, 0, (size_t)d * 8) != cudaSuccess ||
      cudaMemset(b->tp, 0, (size_t)to * b->esz) != cudaSuccess ||
      cudaMemset(b->d_ctl, 0, sizeof(BC) * n) != cudaSuccess)
    return bail(CPALS_E_CUDA);
  *out = b;
  return CPALS_OK;
}

void cpals_batch_destroy(cpals_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->tp) cudaFree(b->tp);
  if (b->dp) cudaFree(b->dp);
  if (b->d_bi) cudaFree(b->d_bi);
  if (b->d_ctl) cudaFree(b->d_ctl);
  if (b->d_ftrace) cudaFree(b->d_ftrace);
  if (b->d_ktrace) cudaFree(b->d_ktrace);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

const char* cpals_batch_last_error(const cpals_batch* b) { return b ? b->err.c_str() : "null batch"; }

cpals_status cpals_batch_set_tensor(cpals_batch* b, int i, const void* data, int dtype, int on_device) {
  if (!b) return CPALS_E_INVALID;
  if (i < 0 || i >= b->n || !data || (dtype != 0 && dtype != 1))
    return b->fail(CPALS_E_INVALID, "bad tensor argument");
  const BI& q = b->bi[i];
  const int64_t n = (int64_t)q.s[0] * q.s[1] * q.s[2];
  const size_t insz = dtype == 0 ? 8 : 4;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  char* dst = static_cast<char*>(b->tp) + (size_t)q.x * b->esz;
  if (insz == b->esz) {
    BCK(cudaMemcpyAsync(dst, data, n * insz, kind, b->stream));
  } else {
    // widen or narrow on the device through a temporary copy
    void* tmp = nullptr;
    if (cudaMalloc(&tmp, n * insz) != cudaSuccess) {
      cudaGetLastError();
      return b->fail(CPALS_E_OOM, "temporary tensor copy");
    }
    cudaError_t e = cudaMemcpyAsync(tmp, data, n * insz, kind, b->stream);
    if (e == cudaSuccess) {
      const int g = (int)std::min<int64_t>(cdiv(n, 256), 4096);
      if (dtype == 0) bconvert_kernel<double, float><<<g, 256, 0, b->stream>>>((const double*)tmp, (float*)dst, n);
      else bconvert_kernel<float, double><<<g, 256, 0, b->stream>>>((const float*)tmp, (double*)dst, n);
      e = cudaStreamSynchronize(b->stream);
    }
    cudaFree(tmp);
    if (e != cudaSuccess) return b->cuda_fail("batch set_tensor", e);
  }
  if (b->esz == 8) bnormx_kernel<double><<<1, 256, 0, b->stream>>>((const double*)dst, n, b->dp + q.sc + 3);
  else bnormx_kernel<float><<<1, 256, 0, b->stream>>>((const float*)dst, n, b->dp + q.sc + 3);
  BCK(cudaGetLastError());
  BCK(cudaStreamSynchronize(b->stream));
  b->have_x[i] = 1;
  return CPALS_OK;
}

cpals_status cpals_batch_init_factors(cpals_batch* b, int i, const double* const* factors) {
  if (!b) return CPALS_E_INVALID;
  if (i < 0 || i >= b->n || !factors) return b->fail(CPALS_E_INVALID, "bad factor argument");
  const BI& q = b->bi[i];
  for (int n = 0; n < 3; n++) {
    if (!factors[n]) return b->fail(CPALS_E_INVALID, "factor pointer is NULL");
    BCK(cudaMemcpyAsync(b->dp + q.a[n], factors[n], (size_t)q.s[n] * q.R * 8, cudaMemcpyHostToDevice,
                        b->stream));
  }
  BCK(cudaStreamSynchronize(b->stream));
  b->have_a[i] = 1;
  return CPALS_OK;
}

cpals_status cpals_batch_run(cpals_batch* b, int max_sweeps, double eps, int use_V, double pp_stop_tol,
                             double* fitness_out, int* sweeps_out, int* status_out, int* kind_trace,
                             double* fitness_trace) {
  if (!b) return CPALS_E_INVALID;
  if (max_sweeps < 1 || !(pp_stop_tol >= 0.0)) return b->fail(CPALS_E_INVALID, "bad run argument");
  for (int i = 0; i < b->n; i++)
    if (!b->have_x[i] || !b->have_a[i])
      return b->fail(CPALS_E_STATE, "instance " + std::to_string(i) + " has no tensor or factors");
  const int64_t cap = (int64_t)b->n * max_sweeps;
  if (cap > b->trace_cap) {
    if (b->d_ftrace) cudaFree(b->d_ftrace);
    if (b->d_ktrace) cudaFree(b->d_ktrace);
    b->d_ftrace = nullptr;
    b->d_ktrace = nullptr;
    b->trace_cap = 0;
    if (cudaMalloc((void**)&b->d_ftrace, cap * 8) != cudaSuccess ||
        cudaMalloc((void**)&b->d_ktrace, cap * 4) != cudaSuccess) {
      cudaGetLastError();
      return b->fail(CPALS_E_OOM, "trace buffers");
    }
    b->trace_cap = cap;
  }
  cpals_status st = b->esz == 8 ? run_impl<double>(b, max_sweeps, eps, use_V != 0, pp_stop_tol)
                                : run_impl<float>(b, max_sweeps, eps, use_V != 0, pp_stop_tol);
  if (st != CPALS_OK) return st;
  std::vector<BC> ctl(b->n);
  BCK(cudaMemcpy(ctl.data(), b->d_ctl, sizeof(BC) * b->n, cudaMemcpyDeviceToHost));
  for (int i = 0; i < b->n; i++) {
    if (sweeps_out) sweeps_out[i] = ctl[i].t;
    if (status_out)
      status_out[i] = (ctl[i].status >> 8) & 1 ? CPALS_E_NUMERIC
                                                : ((ctl[i].status & 0xffff) ? CPALS_E_SINGULAR : CPALS_OK);
    if (fitness_out) BCK(cudaMemcpy(&fitness_out[i], b->dp + b->bi[i].sc, 8, cudaMemcpyDeviceToHost));
  }
  if (kind_trace) BCK(cudaMemcpy(kind_trace, b->d_ktrace, cap * 4, cudaMemcpyDeviceToHost));
  if (fitness_trace) BCK(cudaMemcpy(fitness_trace, b->d_ftrace, cap * 8, cudaMemcpyDeviceToHost));
  return CPALS_OK;
}

cpals_status cpals_batch_get_factors(cpals_batch* b, int i, double* const* out) {
  if (!b) return CPALS_E_INVALID;
  if (i < 0 || i >= b->n || !out) return b->fail(CPALS_E_INVALID, "bad argument");
  const BI& q = b->bi[i];
  for (int n = 0; n < 3; n++) {
    if (!out[n]) return b->fail(CPALS_E_INVALID, "out[n] is NULL");
    BCK(cudaMemcpyAsync(out[n], b->dp + q.a[n], (size_t)q.s[n] * q.R * 8, cudaMemcpyDeviceToHost, b->stream));
  }
  BCK(cudaStreamSynchronize(b->stream));
  return CPALS_OK;
}

cpals_status cpals_batch_stats(const cpals_batch* b, int64_t* launches_per_sweep, int64_t* launches_last_run) {
  if (!b) return CPALS_E_INVALID;
  if (launches_per_sweep) *launches_per_sweep = b->launches_sweep;
  if (launches_last_run) *launches_last_run = b->launches_run;
  return CPALS_OK;
}

cpals_status cpals_batch_tiles(const cpals_batch* b, int* tiles, float* ms, int* from_cache) {
  if (!b) return CPALS_E_INVALID;
  if (!b->tuned) return CPALS_E_STATE;
  for (int st = 0; st < kTuneStages; st++) {
    if (tiles) tiles[st] = b->tile[st];
    if (ms)
      for (int cfg = 0; cfg < kTileCfgs; cfg++) ms[kTileCfgs * st + cfg] = b->tile_ms[st][cfg];
  }
  if (from_cache) *from_cache = b->tile_from_cache ? 1 : 0;
  return CPALS_OK;
}

}  // extern "C"
