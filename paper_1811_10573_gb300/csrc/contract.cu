// SIMT contraction kernels: first-level contraction (float64/float32 CUDA
// cores), multi-TTV of the dimension trees, PP first-order correction,
// Khatri-Rao products and conversions.
//
// Paper: Sec. 2.5 (dimension tree: first level as a matrix product, lower
// levels as batched matrix-vector products sharing r), Sec. 3.2.1 Eq. 3
// (PP update), Sec. 3.2.3 (operator tree).
#include <algorithm>

#include "internal.h"

namespace cpals {

namespace {

constexpr int kThreads = 256;

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ---------------------------------------------------------------- first level
// out_part[z][b][m][r] = sum_{k in chunk z} Xv(b,k,m) * B[k][r]
// Thread (tm, tn) owns rows m = tm + i*THR_M and columns r = tn + j*THR_N
// (strided, so shared-memory reads are conflict free and stores coalesce).
template <typename TX, typename T, bool KMAJOR, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__(kThreads)
gemm_simt_kernel(const TX* __restrict__ X, const T* __restrict__ B, T* __restrict__ out,
                 int64_t batch, int64_t K, int64_t M, int R, int splits, int64_t kchunk,
                 int64_t mtiles) {
  constexpr int THR_N = BN / TN;
  constexpr int THR_M = BM / TM;
  static_assert(THR_N * THR_M == kThreads, "thread layout");
  __shared__ T Xs[BK][BM + 1];
  __shared__ T Bs[BK][BN];

  const int tid = threadIdx.x;
  const int tn = tid % THR_N;
  const int tm = tid / THR_N;
  const int64_t bid = blockIdx.x;
  const int64_t mt = bid % mtiles;
  const int64_t rest = bid / mtiles;
  const int z = (int)(rest % splits);
  const int64_t b = rest / splits;
  const int64_t m0 = mt * BM;
  const int64_t k0 = (int64_t)z * kchunk;
  const int64_t k1 = min(K, k0 + kchunk);
  const TX* Xb = X + b * K * M;

  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; i++)
#pragma unroll
    for (int j = 0; j < TN; j++) acc[i][j] = T(0);
  // warps whose rows are all padding (in the last row tile) skip their FMAs,
  // which frees the FP64 pipe for the SM's other CTAs
  const int wlive = __reduce_max_sync(0xffffffffu, m0 + tm < M ? 1 : 0);

  for (int64_t kk = k0; kk < k1; kk += BK) {
    if (KMAJOR) {
      for (int idx = tid; idx < BK * BM; idx += kThreads) {
        const int k = idx % BK, m = idx / BK;
        const int64_t gk = kk + k, gm = m0 + m;
        Xs[k][m] = (gk < k1 && gm < M) ? T(Xb[gm * K + gk]) : T(0);
      }
    } else {
      for (int idx = tid; idx < BK * BM; idx += kThreads) {
        const int m = idx % BM, k = idx / BM;
        const int64_t gk = kk + k, gm = m0 + m;
        Xs[k][m] = (gk < k1 && gm < M) ? T(Xb[gk * M + gm]) : T(0);
      }
    }
    for (int idx = tid; idx < BK * BN; idx += kThreads) {
      const int r = idx % BN, k = idx / BN;
      const int64_t gk = kk + k;
      Bs[k][r] = (gk < k1 && r < R) ? B[gk * R + r] : T(0);
    }
    __syncthreads();
    if (wlive > 0) {
#pragma unroll
      for (int k = 0; k < BK; k++) {
        T a[TM], bb[TN];
#pragma unroll
        for (int i = 0; i < TM; i++) a[i] = Xs[k][tm + i * THR_M];
#pragma unroll
        for (int j = 0; j < TN; j++) bb[j] = Bs[k][tn + j * THR_N];
#pragma unroll
        for (int i = 0; i < TM; i++)
#pragma unroll
          for (int j = 0; j < TN; j++) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
      }
    }
    __syncthreads();
  }
  T* o = out + ((int64_t)z * batch + b) * M * R;
#pragma unroll
  for (int i = 0; i < TM; i++) {
    const int64_t m = m0 + tm + i * THR_M;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; j++) {
      const int r = tn + j * THR_N;
      if (r < R) o[m * R + r] = acc[i][j];
    }
  }
}

// out[i] = sum_z part[z][i]: 8 warps split the z range (z = w, w+8, ...), then
// a fixed-order combine (deterministic).  32 outputs per CTA, coalesced.
template <typename T>
__global__ void __launch_bounds__(256)
reduce_splits_kernel(const T* __restrict__ part, T* __restrict__ out, int64_t n, int splits) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * 32 + lane;
  T acc = T(0);
  if (i < n) {
#pragma unroll 4
    for (int z = w; z < splits; z += 8) acc += part[(int64_t)z * n + i];
  }
  __shared__ T red[8][33];
  red[w][lane] = acc;
  __syncthreads();
  if (w == 0 && i < n) {
    T sum = red[0][lane];
#pragma unroll
    for (int k = 1; k < 8; k++) sum += red[k][lane];
    out[i] = sum;
  }
}

int grid_for(int64_t n, int threads) {
  return (int)std::min<int64_t>(cdiv(n, threads), 152 * 16);
}

template <typename TX, typename T, bool KM, int BM, int BN, int TM, int TN>
void gemm_launch(const TX* X, const T* B, T* out, T* partials, int64_t batch, int64_t K, int64_t M,
                 int R, int splits, Launch L) {
  constexpr int BK = 16;
  int64_t mtiles = cdiv(M, BM);
  int64_t kchunk = cdiv(cdiv(K, splits), BK) * BK;
  splits = (int)cdiv(K, kchunk);
  T* dst = splits > 1 ? partials : out;
  int64_t blocks = mtiles * batch * splits;
  gemm_simt_kernel<TX, T, KM, BM, BN, BK, TM, TN>
      <<<(unsigned)blocks, kThreads, 0, L.stream>>>(X, B, dst, batch, K, M, R, splits, kchunk,
                                                     mtiles);
  (*L.counter)++;
  if (splits > 1) reduce_splits<T>(partials, out, batch * M * R, splits, L);
}

// ---------------------------------------------------------------- first level, float32, R > 32
// The FP32 pipe (128 FMA per clock per SM) is fed from shared memory, so the
// float32 kernel raises the FMAs per shared load: 128-thread CTAs of 128
// rows x 8*TN columns (TN = ceil(R/8): no padded columns beyond R rounded
// up to 8); thread (tm, tn) owns rows 8 tm .. 8 tm + 7 (two 16-byte shared
// loads per k) and columns tn + 8 j (one 4-byte load each, 8 addresses per
// warp), i.e. 8 TN FMAs for 2 + TN loads.  X arrives in 16-byte loads (k
// contiguous when KMAJOR, else m contiguous; the caller checks the
// alignment).  The next K slab is fetched into registers while the current
// one is multiplied, with two shared buffers and one barrier per slab.
// Measured on GB300 at R = 100, and slower: 16-byte B reads over a padded
// layout (more registers than 2 CTAs per SM leave), 8-deep slabs (global
// latency exposed), a row flip that frees the K-major transpose of its
// 2-way bank conflicts (longer dependency stalls in the multiply loop), and
// K splits into four waves for the few-row launch (partials and their
// reduction cost what the refill gains).  Every output is one fma chain
// over its chunk's k in increasing order, as in gemm_simt_kernel, so the
// results are those of that kernel bit for bit.
constexpr int kF32Threads = 128;
constexpr int kF32BM = 128;
constexpr int kF32BK = 16;

template <bool KMAJOR, int TN>
__global__ void __launch_bounds__(kF32Threads, 2)
gemm_f32_kernel(const float* __restrict__ X, const float* __restrict__ B, float* __restrict__ out,
                int64_t batch, int64_t K, int64_t M, int R, int splits, int64_t kchunk,
                int64_t mtiles) {
  constexpr int NT = kF32Threads, BM = kF32BM, BK = kF32BK, TM = 8, BN = 8 * TN, XS = BM + 4;
  constexpr int NX = BM * BK / 4 / NT;          // 16-byte X loads per thread per slab
  constexpr int NB = (BK * BN + NT - 1) / NT;   // B loads per thread per slab
  constexpr int QPR = BK / 4;                   // 16-byte quads of a K-major row per slab
  static_assert(BK == 8 || BK == 16, "slab depth");
  __shared__ __align__(16) float Xs[2][BK][XS];
  __shared__ __align__(16) float Bs[2][BK][BN];
  const int tid = threadIdx.x, tn = tid & 7, tm = tid >> 3;
  const int64_t bid = blockIdx.x;
  const int64_t mt = bid % mtiles;
  const int64_t rest = bid / mtiles;
  const int z = (int)(rest % splits);
  const int64_t b = rest / splits;
  const int64_t m0 = mt * BM;
  const int64_t k0 = (int64_t)z * kchunk;
  const int64_t k1 = min(K, k0 + kchunk);
  const float* Xb = X + b * K * M;

  float4 xr[NX];
  float br[NB];
  auto fetch = [&](int64_t kk) {
#pragma unroll
    for (int q = 0; q < NX; q++) {
      const int idx = tid + q * NT;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (KMAJOR) {
        const int kq = idx % QPR, m = idx / QPR;   // QPR threads read one row's slab
        const int64_t gk = kk + 4 * kq, gm = m0 + m;
        if (gm < M && gk < k1) v = *reinterpret_cast<const float4*>(Xb + gm * K + gk);
      } else {
        const int m4 = idx & (BM / 4 - 1), k = idx / (BM / 4);
        const int64_t gk = kk + k, gm = m0 + 4 * m4;
        if (gm < M && gk < k1) v = *reinterpret_cast<const float4*>(Xb + gk * M + gm);
      }
      xr[q] = v;
    }
#pragma unroll
    for (int q = 0; q < NB; q++) {
      const int idx = tid + q * NT;
      const int k = idx / BN, r = idx % BN;
      const int64_t gk = kk + k;
      br[q] = (idx < BK * BN && gk < k1 && r < R) ? B[gk * R + r] : 0.f;
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int q = 0; q < NX; q++) {
      const int idx = tid + q * NT;
      if (KMAJOR) {
        const int kq = idx % QPR, m = idx / QPR;
        Xs[buf][4 * kq + 0][m] = xr[q].x;
        Xs[buf][4 * kq + 1][m] = xr[q].y;
        Xs[buf][4 * kq + 2][m] = xr[q].z;
        Xs[buf][4 * kq + 3][m] = xr[q].w;
      } else {
        const int m4 = idx & (BM / 4 - 1), k = idx / (BM / 4);
        *reinterpret_cast<float4*>(&Xs[buf][k][4 * m4]) = xr[q];
      }
    }
#pragma unroll
    for (int q = 0; q < NB; q++) {
      const int idx = tid + q * NT;
      if (idx < BK * BN) Bs[buf][idx / BN][idx % BN] = br[q];
    }
  };

  float acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; i++)
#pragma unroll
    for (int j = 0; j < TN; j++) acc[i][j] = 0.f;
  // warps whose rows are all padding (in the last row tile) skip their FMAs
  const int wlive = __reduce_max_sync(0xffffffffu, m0 + TM * tm < M ? 1 : 0);

  if (k0 < k1) {
    fetch(k0);
    stash(0);
  }
  __syncthreads();
  int buf = 0;
  for (int64_t kk = k0; kk < k1; kk += BK) {
    const bool more = kk + BK < k1;
    if (more) fetch(kk + BK);
    if (wlive > 0) {
#pragma unroll
      for (int k = 0; k < BK; k++) {
        const float4 a0 = *reinterpret_cast<const float4*>(&Xs[buf][k][TM * tm]);
        const float4 a1 = *reinterpret_cast<const float4*>(&Xs[buf][k][TM * tm + 4]);
        const float a[TM] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        float bb[TN];
#pragma unroll
        for (int j = 0; j < TN; j++) bb[j] = Bs[buf][k][tn + 8 * j];
#pragma unroll
        for (int i = 0; i < TM; i++)
#pragma unroll
          for (int j = 0; j < TN; j++) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
      }
    }
    if (more) stash(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
  float* o = out + ((int64_t)z * batch + b) * M * R;
#pragma unroll
  for (int i = 0; i < TM; i++) {
    const int64_t m = m0 + TM * tm + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; j++) {
      const int r = tn + 8 * j;
      if (r < R) o[m * R + r] = acc[i][j];
    }
  }
}

template <bool KM, int TN>
void gemm_f32_launch(const float* X, const float* B, float* out, float* partials, int64_t batch,
                     int64_t K, int64_t M, int R, int splits, Launch L) {
  constexpr int BM = kF32BM, BK = 16;   // K chunks in multiples of 16, as gemm_launch
  const int64_t mtiles = cdiv(M, BM);
  const int64_t kchunk = cdiv(cdiv(K, splits), BK) * BK;
  splits = (int)cdiv(K, kchunk);
  float* dst = splits > 1 ? partials : out;
  const int64_t blocks = mtiles * batch * splits;
  gemm_f32_kernel<KM, TN><<<(unsigned)blocks, kF32Threads, 0, L.stream>>>(X, B, dst, batch, K, M, R,
                                                                        splits, kchunk, mtiles);
  (*L.counter)++;
  if (splits > 1) reduce_splits<float>(partials, out, batch * M * R, splits, L);
}

// The float32 kernel takes R > 32 when the contiguous dimension of X (K for
// the K-major launch, M for the other) allows 16-byte loads.
bool f32_applies(const void* X, int64_t K, int64_t M, int R, bool kmajor) {
  return R > 32 && R <= kMaxRank && (kmajor ? K % 4 == 0 : M % 4 == 0) &&
         (reinterpret_cast<uintptr_t>(X) & 15) == 0;
}

template <bool KM>
void gemm_f32(const float* X, const float* B, float* out, float* partials, int64_t batch, int64_t K,
              int64_t M, int R, int splits, Launch L) {
  switch ((R + 7) / 8) {
    case 5: gemm_f32_launch<KM, 5>(X, B, out, partials, batch, K, M, R, splits, L); break;
    case 6: gemm_f32_launch<KM, 6>(X, B, out, partials, batch, K, M, R, splits, L); break;
    case 7: gemm_f32_launch<KM, 7>(X, B, out, partials, batch, K, M, R, splits, L); break;
    case 8: gemm_f32_launch<KM, 8>(X, B, out, partials, batch, K, M, R, splits, L); break;
    case 9: gemm_f32_launch<KM, 9>(X, B, out, partials, batch, K, M, R, splits, L); break;
    case 10: gemm_f32_launch<KM, 10>(X, B, out, partials, batch, K, M, R, splits, L); break;
    case 11: gemm_f32_launch<KM, 11>(X, B, out, partials, batch, K, M, R, splits, L); break;
    case 12: gemm_f32_launch<KM, 12>(X, B, out, partials, batch, K, M, R, splits, L); break;
    case 13: gemm_f32_launch<KM, 13>(X, B, out, partials, batch, K, M, R, splits, L); break;
    case 14: gemm_f32_launch<KM, 14>(X, B, out, partials, batch, K, M, R, splits, L); break;
    case 15: gemm_f32_launch<KM, 15>(X, B, out, partials, batch, K, M, R, splits, L); break;
    default: gemm_f32_launch<KM, 16>(X, B, out, partials, batch, K, M, R, splits, L); break;
  }
}

// ---------------------------------------------------------------- multi-TTV
// Many outputs per o and a short contracted mode (the operator tree's upper
// levels on small-mode tensors, e.g. 24^5 x R parents): each thread forms
// VEC consecutive outputs over all x in order, so a warp reads 32 VEC
// consecutive values per x and no cross-warp reduction is needed.
template <typename T, int VEC>
__global__ void __launch_bounds__(kThreads)
ttv_cols_kernel(const T* __restrict__ in, const T* __restrict__ A, T* __restrict__ out, int sw,
                int64_t QR, int R, int64_t chunks) {
  const int64_t o = blockIdx.x / chunks;
  const int64_t f = ((blockIdx.x % chunks) * kThreads + threadIdx.x) * VEC;
  if (f >= QR) return;
  const T* base = in + o * sw * QR + f;
  const int r = (int)(f % R);
  if constexpr (VEC == 4) {
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 8
    for (int x = 0; x < sw; x++) {
      const float4 v = *reinterpret_cast<const float4*>(base + (int64_t)x * QR);
      const float4 a = __ldg(reinterpret_cast<const float4*>(A + (int64_t)x * R + r));
      acc.x = fmaf(v.x, a.x, acc.x);
      acc.y = fmaf(v.y, a.y, acc.y);
      acc.z = fmaf(v.z, a.z, acc.z);
      acc.w = fmaf(v.w, a.w, acc.w);
    }
    *reinterpret_cast<float4*>(out + o * QR + f) = acc;
  } else {
    T acc = T(0);
#pragma unroll 8
    for (int x = 0; x < sw; x++) acc = fma(base[(int64_t)x * QR], __ldg(A + (int64_t)x * R + r), acc);
    out[o * QR + f] = acc;
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
ttv_kernel(const T* __restrict__ in, const T* __restrict__ A, T* __restrict__ out, int sw,
           int64_t QR, int R, int64_t chunks) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t o = blockIdx.x / chunks;
  const int64_t c = blockIdx.x % chunks;
  const int64_t f = c * 32 + lane;
  T acc = T(0);
  if (f < QR) {
    const int r = (int)(f % R);
    const T* base = in + o * sw * QR + f;
#pragma unroll 4
    for (int x = w; x < sw; x += 8) acc = fma(base[(int64_t)x * QR], A[(int64_t)x * R + r], acc);
  }
  __shared__ T red[8][33];
  red[w][lane] = acc;
  __syncthreads();
  if (w == 0 && f < QR) {
    T s = red[0][lane];
#pragma unroll
    for (int i = 1; i < 8; i++) s += red[i][lane];
    out[o * QR + f] = s;
  }
}

// float path with 4 outputs per lane (16-byte loads) when R % 4 == 0: a CTA
// takes 128 consecutive (q, r) outputs of one o; 8 warps split x.
__global__ void __launch_bounds__(kThreads)
ttv4_kernel(const float* __restrict__ in, const float* __restrict__ A, float* __restrict__ out,
            int sw, int64_t QR, int R, int64_t chunks) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t o = blockIdx.x / chunks;
  const int64_t c = blockIdx.x % chunks;
  const int64_t f = c * 128 + 4 * lane;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  if (f < QR) {
    const int r = (int)(f % R);
    const float* base = in + o * sw * QR + f;
#pragma unroll 4
    for (int x = w; x < sw; x += 8) {
      const float4 v = *reinterpret_cast<const float4*>(base + (int64_t)x * QR);
      const float4 a = __ldg(reinterpret_cast<const float4*>(A + (int64_t)x * R + r));
      acc.x = fmaf(v.x, a.x, acc.x);
      acc.y = fmaf(v.y, a.y, acc.y);
      acc.z = fmaf(v.z, a.z, acc.z);
      acc.w = fmaf(v.w, a.w, acc.w);
    }
  }
  __shared__ float4 red[8][33];
  red[w][lane] = acc;
  __syncthreads();
  if (w == 0 && f < QR) {
    float4 s = red[0][lane];
#pragma unroll
    for (int i = 1; i < 8; i++) {
      s.x += red[i][lane].x;
      s.y += red[i][lane].y;
      s.z += red[i][lane].z;
      s.w += red[i][lane].w;
    }
    *reinterpret_cast<float4*>(out + o * QR + f) = s;
  }
}

// ---------------------------------------------------------------- PP correction
template <typename T>
struct PPTermsArg {
  PPTerm<T> t[kMaxModes];
  int n;
};

template <typename T>
__global__ void __launch_bounds__(kThreads)
pp_correct_kernel(const T* __restrict__ Mp, PPTermsArg<T> terms, T* __restrict__ out,
                  int64_t total, int R) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t f = (int64_t)blockIdx.x * 32 + lane;
  T acc = T(0);
  if (f < total) {
    const int64_t y = f / R;
    const int r = (int)(f % R);
    for (int t = 0; t < terms.n; t++) {
      const PPTerm<T> tt = terms.t[t];
      const T* base = tt.op + y * tt.ystride + r;
#pragma unroll 4
      for (int x = w; x < tt.sx; x += 8)
        acc = fma(base[(int64_t)x * tt.xstride], tt.dA[(int64_t)x * R + r], acc);
    }
  }
  __shared__ T red[8][33];
  red[w][lane] = acc;
  __syncthreads();
  if (w == 0 && f < total) {
    T s = red[0][lane];
#pragma unroll
    for (int i = 1; i < 8; i++) s += red[i][lane];
    out[f] = Mp[f] + s;
  }
}

// float path when R % 4 == 0: a CTA of 512 threads owns 32 consecutive
// outputs (8 float4 units); lane l of every warp takes unit l % 8 and every
// 64th x starting at 4 * warp + l / 8, so one warp load touches four
// 128-byte runs of the operator.  At 40 registers three CTAs fit on an SM
// (1,250 CTAs for a 400 x 100 mode, 2.7 waves); 256-thread CTAs (1.4 waves)
// measured the same, 31-32 us cold for the 128.6 MB of a mode.  The 64
// partial sums of each output are added in a fixed order (deterministic).
constexpr int kPPThreads = 512;
__global__ void __launch_bounds__(kPPThreads)
pp_correct4_kernel(const float* __restrict__ Mp, PPTermsArg<float> terms, float* __restrict__ out,
                   int64_t total, int R) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int u = lane & 7, xg = 4 * w + (lane >> 3);          // unit, x offset (0..63)
  const int64_t f = (int64_t)blockIdx.x * 32 + 4 * u;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  if (f < total) {
    const int64_t y = f / R;
    const int r = (int)(f % R);
    for (int t = 0; t < terms.n; t++) {
      const PPTerm<float> tt = terms.t[t];
      const float* base = tt.op + y * tt.ystride + r;
      // up to four 16-byte operator loads in flight per thread (the
      // operators are streamed once per sweep: evict-first loads)
      int x = xg;
      for (; x + 192 < tt.sx; x += 256) {
        float4 v[4], a[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
          v[q] = __ldcs(reinterpret_cast<const float4*>(base + (int64_t)(x + 64 * q) * tt.xstride));
          a[q] = __ldg(reinterpret_cast<const float4*>(tt.dA + (int64_t)(x + 64 * q) * R + r));
        }
#pragma unroll
        for (int q = 0; q < 4; q++) {
          acc.x = fmaf(v[q].x, a[q].x, acc.x);
          acc.y = fmaf(v[q].y, a[q].y, acc.y);
          acc.z = fmaf(v[q].z, a[q].z, acc.z);
          acc.w = fmaf(v[q].w, a[q].w, acc.w);
        }
      }
      for (; x < tt.sx; x += 64) {
        const float4 v = __ldcs(reinterpret_cast<const float4*>(base + (int64_t)x * tt.xstride));
        const float4 a = __ldg(reinterpret_cast<const float4*>(tt.dA + (int64_t)x * R + r));
        acc.x = fmaf(v.x, a.x, acc.x);
        acc.y = fmaf(v.y, a.y, acc.y);
        acc.z = fmaf(v.z, a.z, acc.z);
        acc.w = fmaf(v.w, a.w, acc.w);
      }
    }
  }
  __shared__ float4 red[64][9];
  red[xg][u] = acc;
  __syncthreads();
  if (threadIdx.x < 8) {
    const int uu = threadIdx.x;
    const int64_t ff = (int64_t)blockIdx.x * 32 + 4 * uu;
    if (ff < total) {
      float4 sum = red[0][uu];
      for (int i = 1; i < 64; i++) {
        sum.x += red[i][uu].x;
        sum.y += red[i][uu].y;
        sum.z += red[i][uu].z;
        sum.w += red[i][uu].w;
      }
      const float4 m = *reinterpret_cast<const float4*>(Mp + ff);
      *reinterpret_cast<float4*>(out + ff) = make_float4(m.x + sum.x, m.y + sum.y, m.z + sum.z, m.w + sum.w);
    }
  }
}

// ---------------------------------------------------------------- Khatri-Rao
template <typename T>
struct FactorList {
  const T* A[kMaxModes];
  int64_t dims[kMaxModes];
  int n;
};

template <typename T>
__global__ void khatri_rao_kernel(FactorList<T> fl, int R, T* __restrict__ out, int64_t rows) {
  const int64_t n = rows * R;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(i % R);
    int64_t k = i / R;
    T v = T(1);
    for (int j = fl.n - 1; j >= 0; j--) {
      const int64_t ij = k % fl.dims[j];
      k /= fl.dims[j];
      v *= fl.A[j][ij * R + r];
    }
    out[i] = v;
  }
}

// KRP^T in bf16: row r (blockIdx.y) of the transposed Khatri-Rao product.
// Index k = p * s_last + i splits into a prefix p over the leading factors
// and i over the last one.  A CTA takes a range of prefixes: the prefix
// product pf = A_0[i_0][r] * ... * A_{nm-2}[i_{nm-2}][r] (float32, left to
// right) is formed once per prefix, and v = pf * A_{nm-1}[i][r] is rounded to
// bf16 (round to nearest even).  k >= K (padding up to Kstride) is zero.
constexpr int kKrpSmem = 8192;   // floats of the staged last column

__global__ void __launch_bounds__(256)
khatri_rao_bf16_t_kernel(FactorList<float> fl, int R, int64_t K, int64_t Kstride, int64_t nprefix,
                         int64_t pchunk, int64_t ichunk, int64_t lo_off,
                         __nv_bfloat16* __restrict__ outT) {
  __shared__ float col[kKrpSmem];
  const int r = blockIdx.y;
  __nv_bfloat16* o = outT + (int64_t)r * Kstride;
  const int last = fl.n - 1;
  const int64_t sl = fl.dims[last];
  const int64_t nib = (sl + ichunk - 1) / ichunk;      // i-blocks per prefix block
  const int64_t pb = blockIdx.x / nib, ib = blockIdx.x % nib;
  const int64_t p0 = pb * pchunk, p1 = min(nprefix, p0 + pchunk);
  const int64_t i0 = ib * ichunk, i1 = min(sl, i0 + ichunk);
  // zero padding k in [K, Kstride): taken by the first CTA of the row
  if (blockIdx.x == 0)
    for (int64_t k = K + threadIdx.x; k < Kstride; k += blockDim.x) {
      o[k] = __float2bfloat16_rn(0.f);
      o[lo_off + k] = __float2bfloat16_rn(0.f);
    }
  if (r >= R) {
    for (int64_t p = p0; p < p1; p++)
      for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        o[p * sl + i] = __float2bfloat16_rn(0.f);
        o[lo_off + p * sl + i] = __float2bfloat16_rn(0.f);
      }
    return;
  }
  const bool staged = (i1 - i0) <= kKrpSmem;
  if (staged)
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) col[i - i0] = fl.A[last][i * R + r];
  __syncthreads();
  for (int64_t p = p0; p < p1; p++) {
    float pf = 1.f;
    if (last > 0) {
      // decode p into the leading indices (last leading factor fastest)
      uint32_t idx[kMaxModes];
      uint32_t q = (uint32_t)p;
      for (int j = last - 1; j >= 0; j--) {
        const uint32_t d = (uint32_t)fl.dims[j];
        idx[j] = q % d;
        q /= d;
      }
      pf = fl.A[0][(int64_t)idx[0] * R + r];
      for (int j = 1; j < last; j++) pf *= fl.A[j][(int64_t)idx[j] * R + r];
    }
    __nv_bfloat16* op = o + p * sl;
    __nv_bfloat16* opl = op + lo_off;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
      const float a = staged ? col[i - i0] : fl.A[last][i * R + r];
      const float v = last > 0 ? pf * a : a;
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      op[i] = h;
      opl[i] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
  }
}

template <typename TS, typename TD>
__global__ void convert_kernel(const TS* __restrict__ s, TD* __restrict__ d, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    d[i] = (TD)s[i];
}

template <>
__global__ void convert_kernel<float, __nv_bfloat16>(const float* __restrict__ s,
                                                     __nv_bfloat16* __restrict__ d, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    d[i] = __float2bfloat16_rn(s[i]);
}

template <typename TX>
__global__ void sumsq_part_kernel(const TX* __restrict__ x, int64_t n, double* __restrict__ part) {
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)x[i];
    acc = fma(v, v, acc);
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void sum_parts_kernel(const double* __restrict__ part, int n, double* __restrict__ out) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) acc += part[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}

}  // namespace

// ---------------------------------------------------------------- host wrappers
template <typename T>
void reduce_splits(const T* part, T* out, int64_t n, int splits, Launch L) {
  reduce_splits_kernel<T><<<(unsigned)cdiv(n, 32), 256, 0, L.stream>>>(part, out, n, splits);
  (*L.counter)++;
}

// Rows per tile of the configuration gemm_simt picks for (M, R, kmajor).
static int64_t gemm_simt_bm(int64_t M, int R, bool kmajor) {
  if (!kmajor && M <= 32 && R <= 64) return 32;
  return R <= 32 ? 128 : 64;
}

int gemm_simt_splits(int64_t batch, int64_t K, int64_t M, int R, bool kmajor, int64_t cap,
                     int min_blocks) {
  const int64_t base = cdiv(M, gemm_simt_bm(M, R, kmajor)) * batch;
  if (base >= min_blocks) return 1;
  int64_t sp = cdiv(min_blocks, base);
  sp = std::min<int64_t>(sp, std::max<int64_t>(1, K / 64));      // at least 64 k per split
  sp = std::min<int64_t>(sp, cap / std::max<int64_t>(1, batch * M * R));
  return (int)std::max<int64_t>(sp, 1);
}

// float64 contractions with R > 32: 64-row tiles whose column tile is R
// rounded up to a multiple of 8 (8 thread columns of TN = ceil(R/8) each), or
// R itself when R = 4 (mod 8) above 64, so the FP64 pipe, the bound of these
// kernels, runs few or no padded FMAs (R = 100: 100 columns instead of 128).
// Each output's k order is the same as with any other tile.
// R = 4 (mod 8) above 64 (R = 100 would pad 4 columns to 104): 64-row tiles
// of exactly R columns, 4 thread columns of R/4 each and 64 thread rows of
// one row.
constexpr bool exact4(int R) { return R > 64 && R % 8 == 4; }

template <typename TX, typename T, bool KM>
void gemm_exact_launch(const TX* X, const T* B, T* out, T* partials, int64_t batch, int64_t K,
                       int64_t M, int R, int splits, Launch L) {
  if (exact4(R)) {
    switch (R) {
      case 68: gemm_launch<TX, T, KM, 64, 68, 1, 17>(X, B, out, partials, batch, K, M, R, splits, L); return;
      case 76: gemm_launch<TX, T, KM, 64, 76, 1, 19>(X, B, out, partials, batch, K, M, R, splits, L); return;
      case 84: gemm_launch<TX, T, KM, 64, 84, 1, 21>(X, B, out, partials, batch, K, M, R, splits, L); return;
      case 92: gemm_launch<TX, T, KM, 64, 92, 1, 23>(X, B, out, partials, batch, K, M, R, splits, L); return;
      case 100: gemm_launch<TX, T, KM, 64, 100, 1, 25>(X, B, out, partials, batch, K, M, R, splits, L); return;
      case 108: gemm_launch<TX, T, KM, 64, 108, 1, 27>(X, B, out, partials, batch, K, M, R, splits, L); return;
      case 116: gemm_launch<TX, T, KM, 64, 116, 1, 29>(X, B, out, partials, batch, K, M, R, splits, L); return;
      default: gemm_launch<TX, T, KM, 64, 124, 1, 31>(X, B, out, partials, batch, K, M, R, splits, L); return;
    }
  }
  switch ((R + 7) / 8) {
    case 5: gemm_launch<TX, T, KM, 64, 40, 2, 5>(X, B, out, partials, batch, K, M, R, splits, L); break;
    case 6: gemm_launch<TX, T, KM, 64, 48, 2, 6>(X, B, out, partials, batch, K, M, R, splits, L); break;
    case 7: gemm_launch<TX, T, KM, 64, 56, 2, 7>(X, B, out, partials, batch, K, M, R, splits, L); break;
    case 8: gemm_launch<TX, T, KM, 64, 64, 2, 8>(X, B, out, partials, batch, K, M, R, splits, L); break;
    case 9: gemm_launch<TX, T, KM, 64, 72, 2, 9>(X, B, out, partials, batch, K, M, R, splits, L); break;
    case 10: gemm_launch<TX, T, KM, 64, 80, 2, 10>(X, B, out, partials, batch, K, M, R, splits, L); break;
    case 11: gemm_launch<TX, T, KM, 64, 88, 2, 11>(X, B, out, partials, batch, K, M, R, splits, L); break;
    case 12: gemm_launch<TX, T, KM, 64, 96, 2, 12>(X, B, out, partials, batch, K, M, R, splits, L); break;
    case 13: gemm_launch<TX, T, KM, 64, 104, 2, 13>(X, B, out, partials, batch, K, M, R, splits, L); break;
    case 14: gemm_launch<TX, T, KM, 64, 112, 2, 14>(X, B, out, partials, batch, K, M, R, splits, L); break;
    case 15: gemm_launch<TX, T, KM, 64, 120, 2, 15>(X, B, out, partials, batch, K, M, R, splits, L); break;
    default: gemm_launch<TX, T, KM, 64, 128, 2, 16>(X, B, out, partials, batch, K, M, R, splits, L); break;
  }
}

// Resident CTAs per SM of the float64 configuration gemm_exact_cols launches
// for R (queried once per configuration).
template <typename TX, bool KM, int BN, int TN, int TM = 2>
int exact_cols_occ() {
  static int occ = 0;
  if (occ == 0) {
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &o, gemm_simt_kernel<TX, double, KM, 64, BN, 16, TM, TN>, kThreads, 0) != cudaSuccess ||
        o < 1) {
      cudaGetLastError();
      o = 1;
    }
    occ = o;
  }
  return occ;
}

template <typename TX, bool KM>
int exact_cols_occ_for(int R) {
  if (exact4(R)) {
    switch (R) {
      case 68: return exact_cols_occ<TX, KM, 68, 17, 1>();
      case 76: return exact_cols_occ<TX, KM, 76, 19, 1>();
      case 84: return exact_cols_occ<TX, KM, 84, 21, 1>();
      case 92: return exact_cols_occ<TX, KM, 92, 23, 1>();
      case 100: return exact_cols_occ<TX, KM, 100, 25, 1>();
      case 108: return exact_cols_occ<TX, KM, 108, 27, 1>();
      case 116: return exact_cols_occ<TX, KM, 116, 29, 1>();
      default: return exact_cols_occ<TX, KM, 124, 31, 1>();
    }
  }
  switch ((R + 7) / 8) {
    case 5: return exact_cols_occ<TX, KM, 40, 5>();
    case 6: return exact_cols_occ<TX, KM, 48, 6>();
    case 7: return exact_cols_occ<TX, KM, 56, 7>();
    case 8: return exact_cols_occ<TX, KM, 64, 8>();
    case 9: return exact_cols_occ<TX, KM, 72, 9>();
    case 10: return exact_cols_occ<TX, KM, 80, 10>();
    case 11: return exact_cols_occ<TX, KM, 88, 11>();
    case 12: return exact_cols_occ<TX, KM, 96, 12>();
    case 13: return exact_cols_occ<TX, KM, 104, 13>();
    case 14: return exact_cols_occ<TX, KM, 112, 14>();
    case 15: return exact_cols_occ<TX, KM, 120, 15>();
    default: return exact_cols_occ<TX, KM, 128, 16>();
  }
}

int sm_count() {
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
      cudaGetLastError();
      return 0;
    }
    nsm = n;
  }
  return nsm;
}

// A K-major launch of one batch whose 64-row tiles fill w whole waves of
// resident CTAs and part of one more (R = 100 at 400^3: 2,500 tiles, 8.2
// waves of 304) runs as two launches: the whole waves, then the remaining
// rows with K split so that they fill one wave, their partials summed by
// reduce_splits (part_cap: values the partials buffer holds; 0 keeps one
// launch).  The last wave then takes a fraction of a CTA's time instead of
// a whole one with most SMs idle.
template <typename TX, typename T, bool KM>
void gemm_exact_cols(const TX* X, const T* B, T* out, T* partials, int64_t batch, int64_t K,
                     int64_t M, int R, int splits, Launch L, int64_t part_cap) {
  if (KM && batch == 1 && splits == 1 && part_cap > 0) {
    const int64_t wave = (int64_t)exact_cols_occ_for<TX, true>(R) * sm_count();
    const int64_t tiles = cdiv(M, 64);
    const int64_t full = wave > 0 ? tiles / wave * wave : 0;
    if (full > 0 && full < tiles) {
      const int64_t rows = M - full * 64;
      int64_t sp = wave / (tiles - full);
      sp = std::min<int64_t>(sp, K / 16);
      sp = std::min<int64_t>(sp, part_cap / std::max<int64_t>(1, rows * R));
      while (sp > 1 && cdiv(K, cdiv(cdiv(K, sp), 16) * 16) != sp) sp--;
      if (sp >= 2) {
        gemm_exact_launch<TX, T, KM>(X, B, out, partials, 1, K, full * 64, R, 1, L);
        gemm_exact_launch<TX, T, KM>(X + full * 64 * K, B, out + full * 64 * R, partials, 1, K, rows, R,
                                     (int)sp, L);
        return;
      }
    }
  }
  gemm_exact_launch<TX, T, KM>(X, B, out, partials, batch, K, M, R, splits, L);
}

template <typename TX, typename T>
void gemm_simt(const TX* X, const T* B, T* out, T* partials, int64_t batch, int64_t K, int64_t M,
               int R, bool kmajor, int splits, Launch L, int64_t part_cap) {
  if (splits < 1) splits = 1;
  if constexpr (sizeof(T) == 4 && sizeof(TX) == 4) {
    if (f32_applies(X, K, M, R, kmajor)) {
      if (kmajor) gemm_f32<true>(X, B, out, partials, batch, K, M, R, splits, L);
      else gemm_f32<false>(X, B, out, partials, batch, K, M, R, splits, L);
      return;
    }
  }
  if constexpr (sizeof(T) == 8) {
    if (R > 32 && gemm_simt_bm(M, R, kmajor) == 64) {
      if (kmajor) gemm_exact_cols<TX, T, true>(X, B, out, partials, batch, K, M, R, splits, L, part_cap);
      else gemm_exact_cols<TX, T, false>(X, B, out, partials, batch, K, M, R, splits, L, part_cap);
      return;
    }
  }
  if (gemm_simt_bm(M, R, kmajor) == 32) {
    // few rows per batch (batched lower-level contractions): 32-row tiles
    if (R <= 32) gemm_launch<TX, T, false, 32, 32, 2, 2>(X, B, out, partials, batch, K, M, R, splits, L);
    else gemm_launch<TX, T, false, 32, 64, 2, 4>(X, B, out, partials, batch, K, M, R, splits, L);
  } else if (R <= 16) {
    // narrower column tiles for small R (no padded FMAs on the FP64 pipe)
    if (kmajor) gemm_launch<TX, T, true, 128, 16, 8, 1>(X, B, out, partials, batch, K, M, R, splits, L);
    else gemm_launch<TX, T, false, 128, 16, 8, 1>(X, B, out, partials, batch, K, M, R, splits, L);
  } else if (R <= 24) {
    if (kmajor) gemm_launch<TX, T, true, 128, 24, 4, 3>(X, B, out, partials, batch, K, M, R, splits, L);
    else gemm_launch<TX, T, false, 128, 24, 4, 3>(X, B, out, partials, batch, K, M, R, splits, L);
  } else if (R <= 32) {
    if (kmajor) gemm_launch<TX, T, true, 128, 32, 8, 2>(X, B, out, partials, batch, K, M, R, splits, L);
    else gemm_launch<TX, T, false, 128, 32, 8, 2>(X, B, out, partials, batch, K, M, R, splits, L);
  } else if (R <= 64) {
    if (kmajor) gemm_launch<TX, T, true, 64, 64, 4, 4>(X, B, out, partials, batch, K, M, R, splits, L);
    else gemm_launch<TX, T, false, 64, 64, 4, 4>(X, B, out, partials, batch, K, M, R, splits, L);
  } else {
    if (kmajor) gemm_launch<TX, T, true, 64, 128, 4, 8>(X, B, out, partials, batch, K, M, R, splits, L);
    else gemm_launch<TX, T, false, 64, 128, 4, 8>(X, B, out, partials, batch, K, M, R, splits, L);
  }
}

int gemm_simt_wave_splits(int64_t batch, int64_t K, int64_t M, int R, bool kmajor, size_t esz,
                          int64_t cap) {
  if (esz != 8) return 0;
  int nsm = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) {
    cudaGetLastError();
    return 0;
  }
  if (R <= 32 || gemm_simt_bm(M, R, kmajor) != 64) {
    // small float64 contractions: a CTA's time is its tile times its K chunk
    // on one SM's FP64 pipe, so split K until every SM has a CTA, down to
    // one 16-wide K step per split
    const int64_t tiles = cdiv(M, gemm_simt_bm(M, R, kmajor)) * batch;
    if (tiles >= nsm) return 1;
    int64_t sp = std::min<int64_t>(cdiv(nsm, tiles), cdiv(K, 16));
    sp = std::min<int64_t>(sp, cap / std::max<int64_t>(1, batch * M * R));
    while (sp > 1 && cdiv(K, cdiv(cdiv(K, sp), 16) * 16) != sp) sp--;
    return (int)std::max<int64_t>(sp, 1);
  }
  const int occ = kmajor ? exact_cols_occ_for<double, true>(R) : exact_cols_occ_for<double, false>(R);
  const int64_t wave = (int64_t)occ * nsm;
  const int64_t tiles = cdiv(M, 64) * batch;
  if (tiles >= wave) return 1;
  // about four waves: the CTAs of a partly padded row tile finish early (their
  // padding warps skip the FMAs) and the block scheduler refills their SMs
  int64_t sp = 4 * wave / tiles;
  sp = std::min<int64_t>(sp, std::max<int64_t>(1, K / 256));      // at least 256 k per split
  sp = std::min<int64_t>(sp, cap / std::max<int64_t>(1, batch * M * R));
  // the kernel rounds the chunk up to 16 k: keep only counts it runs as given
  while (sp > 1 && cdiv(K, cdiv(cdiv(K, sp), 16) * 16) != sp) sp--;
  return (int)std::max<int64_t>(sp, 1);
}

template <typename T>
void ttv(const T* in, const T* A, T* out, int64_t outer, int sw, int64_t inner, int R, Launch L) {
  const int64_t QR = inner * R;
  if (sw <= 64 && outer * QR >= (int64_t)152 * 64 * kThreads) {
    // enough outputs for every thread to own some: no split of x
    if (sizeof(T) == 4 && R % 4 == 0) {
      const int64_t chunks = cdiv(QR, 4 * kThreads);
      ttv_cols_kernel<float, 4><<<(unsigned)(outer * chunks), kThreads, 0, L.stream>>>(
          (const float*)in, (const float*)A, (float*)out, sw, QR, R, chunks);
    } else {
      const int64_t chunks = cdiv(QR, kThreads);
      ttv_cols_kernel<T, 1><<<(unsigned)(outer * chunks), kThreads, 0, L.stream>>>(in, A, out, sw, QR, R,
                                                                                  chunks);
    }
    (*L.counter)++;
    return;
  }
  if (sizeof(T) == 4 && R % 4 == 0) {
    const int64_t chunks = cdiv(QR, 128);
    ttv4_kernel<<<(unsigned)(outer * chunks), kThreads, 0, L.stream>>>(
        (const float*)in, (const float*)A, (float*)out, sw, QR, R, chunks);
    (*L.counter)++;
    return;
  }
  const int64_t chunks = cdiv(QR, 32);
  ttv_kernel<T><<<(unsigned)(outer * chunks), kThreads, 0, L.stream>>>(in, A, out, sw, QR, R, chunks);
  (*L.counter)++;
}

template <typename T>
void pp_correct(const T* Mp, const PPTerm<T>* terms, int nterms, T* out, int sy, int R, Launch L) {
  PPTermsArg<T> a;
  a.n = nterms;
  for (int i = 0; i < nterms; i++) a.t[i] = terms[i];
  const int64_t total = (int64_t)sy * R;
  if (sizeof(T) == 4 && R % 4 == 0) {
    pp_correct4_kernel<<<(unsigned)cdiv(total, 32), kPPThreads, 0, L.stream>>>(
        (const float*)Mp, *reinterpret_cast<PPTermsArg<float>*>(&a), (float*)out, total, R);
    (*L.counter)++;
    return;
  }
  pp_correct_kernel<T><<<(unsigned)cdiv(total, 32), kThreads, 0, L.stream>>>(Mp, a, out, total, R);
  (*L.counter)++;
}

template <typename T>
void khatri_rao(const T* const* A, const int64_t* dims, int nm, int R, T* out, Launch L) {
  FactorList<T> fl;
  fl.n = nm;
  int64_t rows = 1;
  for (int i = 0; i < nm; i++) {
    fl.A[i] = A[i];
    fl.dims[i] = dims[i];
    rows *= dims[i];
  }
  khatri_rao_kernel<T><<<grid_for(rows * R, 256), 256, 0, L.stream>>>(fl, R, out, rows);
  (*L.counter)++;
}

void khatri_rao_bf16_t(const float* const* A, const int64_t* dims, int nm, int R, int Rpad,
                       int64_t Kstride, __nv_bfloat16* outT, Launch L) {
  FactorList<float> fl;
  fl.n = nm;
  int64_t K = 1;
  for (int i = 0; i < nm; i++) {
    fl.A[i] = A[i];
    fl.dims[i] = dims[i];
    K *= dims[i];
  }
  const int64_t sl = dims[nm - 1];
  const int64_t nprefix = K / sl;
  const int64_t ichunk = std::min<int64_t>(sl, kKrpSmem);
  const int64_t pchunk = std::max<int64_t>(1, 4096 / ichunk);
  const int64_t blocks = cdiv(nprefix, pchunk) * cdiv(sl, ichunk);
  dim3 grid((unsigned)blocks, (unsigned)Rpad);
  khatri_rao_bf16_t_kernel<<<grid, 256, 0, L.stream>>>(fl, R, K, Kstride, nprefix, pchunk, ichunk,
                                                      (int64_t)Rpad * Kstride, outT);
  (*L.counter)++;
}

template <typename TS, typename TD>
void convert(const TS* src, TD* dst, int64_t n, Launch L) {
  convert_kernel<TS, TD><<<grid_for(n, 256), 256, 0, L.stream>>>(src, dst, n);
  (*L.counter)++;
}

template <typename TX>
void sumsq(const TX* x, int64_t n, double* partials, double* out, Launch L) {
  const int blocks = 1024;
  sumsq_part_kernel<TX><<<blocks, 256, 0, L.stream>>>(x, n, partials);
  sum_parts_kernel<<<1, 256, 0, L.stream>>>(partials, blocks, out);
  (*L.counter) += 2;
}

// ---------------------------------------------------------------- instantiations
template void reduce_splits<float>(const float*, float*, int64_t, int, Launch);
template void reduce_splits<double>(const double*, double*, int64_t, int, Launch);
template void gemm_simt<double, double>(const double*, const double*, double*, double*, int64_t,
                                        int64_t, int64_t, int, bool, int, Launch, int64_t);
template void gemm_simt<float, float>(const float*, const float*, float*, float*, int64_t, int64_t,
                                      int64_t, int, bool, int, Launch, int64_t);
template void ttv<double>(const double*, const double*, double*, int64_t, int, int64_t, int, Launch);
template void ttv<float>(const float*, const float*, float*, int64_t, int, int64_t, int, Launch);
template void pp_correct<double>(const double*, const PPTerm<double>*, int, double*, int, int, Launch);
template void pp_correct<float>(const float*, const PPTerm<float>*, int, float*, int, int, Launch);
template void khatri_rao<double>(const double* const*, const int64_t*, int, int, double*, Launch);
template void khatri_rao<float>(const float* const*, const int64_t*, int, int, float*, Launch);
template void convert<double, float>(const double*, float*, int64_t, Launch);
template void convert<float, double>(const float*, double*, int64_t, Launch);
template void convert<double, double>(const double*, double*, int64_t, Launch);
template void convert<float, float>(const float*, float*, int64_t, Launch);
template void convert<float, __nv_bfloat16>(const float*, __nv_bfloat16*, int64_t, Launch);
template void sumsq<double>(const double*, int64_t, double*, double*, Launch);
template void sumsq<float>(const float*, int64_t, double*, double*, Launch);

}  // namespace cpals
