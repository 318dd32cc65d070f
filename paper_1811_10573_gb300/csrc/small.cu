// Float64 kernels of the normal-equation update (Sec. 2.3, Algorithm 1 lines
// 5-10, Algorithm 3 lines 11-17) and the fitness (Sec. 5).  R <= 128.
#include <algorithm>

#include "internal.h"

namespace cpals {

namespace {

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ---------------------------------------------------------------- Gamma + Cholesky (+ Z)
// One CTA: Gamma^(n) = Hadamard product of S^(k), k != n, then a right-looking
// Cholesky Gamma = L L^T in shared memory.  With useV also
// Z = sum_{i<j; i,j != n} W_i * W_j * (*_{k not in {i,j,n}} S_k) (Eq. 3's
// V terms: sum V^(n,i,j) = A^(n) Z).
__global__ void __launch_bounds__(512)
gamma_chol_kernel(const double* __restrict__ S, const double* __restrict__ W, int N, int n, int R,
                  double* __restrict__ Lout, double* __restrict__ Z, int useV,
                  int* __restrict__ status) {
  extern __shared__ double G[];
  __shared__ int bad;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int RR = R * R;
  for (int idx = tid; idx < RR; idx += nt) {
    double g = 1.0;
    for (int k = 0; k < N; k++)
      if (k != n) g *= S[(int64_t)k * RR + idx];
    G[idx] = g;
    if (useV) {
      double z = 0.0;
      for (int i = 0; i < N; i++) {
        if (i == n) continue;
        for (int j = i + 1; j < N; j++) {
          if (j == n) continue;
          double h = W[(int64_t)i * RR + idx] * W[(int64_t)j * RR + idx];
          for (int k = 0; k < N; k++)
            if (k != i && k != j && k != n) h *= S[(int64_t)k * RR + idx];
          z += h;
        }
      }
      Z[idx] = z;
    }
  }
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int k = 0; k < R; k++) {
    const double piv = G[k * R + k];
    if (!(piv > 0.0) || !isfinite(piv)) {
      if (tid == 0) bad = 1;
      break;
    }
    const double l = sqrt(piv);
    const double il = 1.0 / l;
    __syncthreads();
    if (tid == 0) G[k * R + k] = l;
    for (int i = k + 1 + tid; i < R; i += nt) G[i * R + k] *= il;
    __syncthreads();
    const int m = R - k - 1;
    for (int idx = tid; idx < m * m; idx += nt) {
      const int i = k + 1 + idx / m, j = k + 1 + idx % m;
      if (j <= i) G[i * R + j] -= G[i * R + k] * G[j * R + k];
    }
    __syncthreads();
  }
  __syncthreads();
  if (bad) {
    if (tid == 0) atomicOr(status, 1 << n);
    return;
  }
  for (int idx = tid; idx < RR; idx += nt) {
    const int i = idx / R, j = idx % R;
    Lout[idx] = (j <= i) ? G[idx] : 0.0;
  }
}

// rhs2[y][r] = rhs[y][r] + sum_k A[y][k] Z[k][r]  (second-order PP terms)
template <typename T>
__global__ void vterm_kernel(const T* __restrict__ rhs, const double* __restrict__ A,
                             const double* __restrict__ Z, double* __restrict__ out, int s, int R) {
  const int64_t n = (int64_t)s * R;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t y = i / R;
    const int r = (int)(i % R);
    double acc = (double)rhs[i];
    for (int k = 0; k < R; k++) acc = fma(A[y * R + k], Z[k * R + r], acc);
    out[i] = acc;
  }
}

// ---------------------------------------------------------------- row solves
constexpr int kChunks = kMaxRank / 32;

__device__ __forceinline__ double pick(const double (&v)[kChunks], int c) {
  double out = v[0];
#pragma unroll
  for (int i = 1; i < kChunks; i++)
    if (c == i) out = v[i];
  return out;
}
__device__ __forceinline__ void put(double (&v)[kChunks], int c, double x) {
#pragma unroll
  for (int i = 0; i < kChunks; i++)
    if (c == i) v[i] = x;
}

// One warp per row y: forward substitution L z = b, back substitution
// L^T a = z, i.e. a = b Gamma^{-1} (two triangular solves per row).
template <typename TR, typename T>
__global__ void __launch_bounds__(128)
solve_rows_kernel(const TR* __restrict__ rhs, double* __restrict__ A,
                  const double* __restrict__ Aref, double* __restrict__ dA,
                  const double* __restrict__ Lg, T* __restrict__ Ac, T* __restrict__ dAc,
                  double* __restrict__ rownorm, int s, int R, int n, const int* __restrict__ status) {
  extern __shared__ double Ls[];   // R*R lower factor, then R inverse diagonals
  double* inv = Ls + R * R;
  const bool failed = (status[0] >> n) & 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  if (!failed) {
    for (int idx = threadIdx.x; idx < R * R; idx += blockDim.x) Ls[idx] = Lg[idx];
    __syncthreads();
    for (int i = threadIdx.x; i < R; i += blockDim.x) inv[i] = 1.0 / Ls[i * R + i];
    __syncthreads();
  }
  for (int y = blockIdx.x * nw + warp; y < s; y += gridDim.x * nw) {
    double b[kChunks], old[kChunks];
#pragma unroll
    for (int c = 0; c < kChunks; c++) {
      const int r = lane + 32 * c;
      old[c] = r < R ? A[(int64_t)y * R + r] : 0.0;
      b[c] = r < R ? (double)rhs[(int64_t)y * R + r] : 0.0;
    }
    if (failed) {
#pragma unroll
      for (int c = 0; c < kChunks; c++) b[c] = old[c];
    } else {
      for (int i = 0; i < R; i++) {
        const int ci = i >> 5, li = i & 31;
        const double zi = __shfl_sync(0xffffffffu, pick(b, ci), li) * inv[i];
        if (lane == li) put(b, ci, zi);
#pragma unroll
        for (int c = 0; c < kChunks; c++) {
          const int r = lane + 32 * c;
          if (r > i && r < R) b[c] = fma(-Ls[r * R + i], zi, b[c]);
        }
      }
      for (int i = R - 1; i >= 0; i--) {
        const int ci = i >> 5, li = i & 31;
        const double ai = __shfl_sync(0xffffffffu, pick(b, ci), li) * inv[i];
        if (lane == li) put(b, ci, ai);
#pragma unroll
        for (int c = 0; c < kChunks; c++) {
          const int r = lane + 32 * c;
          if (r < i) b[c] = fma(-Ls[i * R + r], ai, b[c]);
        }
      }
    }
    double nd = 0.0, na = 0.0;
#pragma unroll
    for (int c = 0; c < kChunks; c++) {
      const int r = lane + 32 * c;
      if (r < R) {
        const int64_t o = (int64_t)y * R + r;
        const double ref = Aref ? Aref[o] : old[c];
        const double d = failed ? dA[o] : b[c] - ref;
        A[o] = b[c];
        dA[o] = d;
        Ac[o] = (T)b[c];
        dAc[o] = (T)d;
        nd = fma(d, d, nd);
        na = fma(b[c], b[c], na);
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      nd += __shfl_xor_sync(0xffffffffu, nd, off);
      na += __shfl_xor_sync(0xffffffffu, na, off);
    }
    if (lane == 0) {
      rownorm[2 * y] = nd;
      rownorm[2 * y + 1] = na;
    }
  }
}

// ---------------------------------------------------------------- Grams
// partials[z][tile][32][32]: tile t < ntS is an upper block (ti <= tj) of A^T A,
// the rest are blocks of A^T dA.  Rows [z*chunk, (z+1)*chunk).
__global__ void __launch_bounds__(256)
gram_part_kernel(const double* __restrict__ A, const double* __restrict__ dA, int s, int R,
                 int nb, int ntS, int ntiles, int chunk, double* __restrict__ part) {
  const int t = blockIdx.x % ntiles;
  const int z = blockIdx.x / ntiles;
  int ti, tj;
  const double* Bm;
  if (t < ntS) {
    int tt = t;
    ti = 0;
    while (tt >= nb - ti) { tt -= nb - ti; ti++; }
    tj = ti + tt;
    Bm = A;
  } else {
    ti = (t - ntS) / nb;
    tj = (t - ntS) % nb;
    Bm = dA;
  }
  __shared__ double As[32][33], Bs[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const int y0 = z * chunk, y1 = min(s, y0 + chunk);
  for (int yb = y0; yb < y1; yb += 32) {
    for (int idx = threadIdx.x; idx < 32 * 32; idx += 256) {
      const int yy = idx / 32, c = idx % 32;
      const int y = yb + yy;
      const int ci = ti * 32 + c, cj = tj * 32 + c;
      As[yy][c] = (y < y1 && ci < R) ? A[(int64_t)y * R + ci] : 0.0;
      Bs[yy][c] = (y < y1 && cj < R) ? Bm[(int64_t)y * R + cj] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int yy = 0; yy < 32; yy++) {
      const double bj = Bs[yy][tx];
#pragma unroll
      for (int q = 0; q < 4; q++) acc[q] = fma(As[yy][ty + 8 * q], bj, acc[q]);
    }
    __syncthreads();
  }
  double* p = part + ((int64_t)z * ntiles + t) * 1024;
#pragma unroll
  for (int q = 0; q < 4; q++) p[(ty + 8 * q) * 32 + tx] = acc[q];
}

__global__ void gram_reduce_kernel(const double* __restrict__ part, int R, int nb, int ntS,
                                   int ntiles, int splits, bool withW, double* __restrict__ S,
                                   double* __restrict__ W, const double* __restrict__ rownorm,
                                   int s, double* __restrict__ scal) {
  const int nt_use = withW ? ntiles : ntS;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nt_use * 1024;
       idx += gridDim.x * blockDim.x) {
    const int t = idx / 1024, e = idx % 1024;
    double acc = 0.0;
    for (int z = 0; z < splits; z++) acc += part[((int64_t)z * ntiles + t) * 1024 + e];
    const int li = e / 32, lj = e % 32;
    if (t < ntS) {
      int tt = t, ti = 0;
      while (tt >= nb - ti) { tt -= nb - ti; ti++; }
      const int tj = ti + tt;
      const int i = ti * 32 + li, j = tj * 32 + lj;
      if (i < R && j < R) {
        S[i * R + j] = acc;
        S[j * R + i] = acc;
      }
    } else {
      const int ti = (t - ntS) / nb, tj = (t - ntS) % nb;
      const int i = ti * 32 + li, j = tj * 32 + lj;
      if (i < R && j < R) W[i * R + j] = acc;
    }
  }
  if (blockIdx.x == 0) {
    __shared__ double rd[256], ra[256];
    double a = 0.0, b = 0.0;
    for (int y = threadIdx.x; y < s; y += blockDim.x) {
      a += rownorm[2 * y];
      b += rownorm[2 * y + 1];
    }
    rd[threadIdx.x] = a;
    ra[threadIdx.x] = b;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
      if ((int)threadIdx.x < st) {
        rd[threadIdx.x] += rd[threadIdx.x + st];
        ra[threadIdx.x] += ra[threadIdx.x + st];
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      scal[0] = rd[0];
      scal[1] = ra[0];
    }
  }
}

// ---------------------------------------------------------------- fitness
template <typename T>
__global__ void fitness_part_kernel(const T* __restrict__ rhs, const double* __restrict__ A,
                                    const double* __restrict__ S, int N, int R, int s,
                                    double* __restrict__ part) {
  const int64_t n1 = (int64_t)s * R;
  const int RR = R * R;
  double a = 0.0, b = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n1;
       i += (int64_t)gridDim.x * blockDim.x)
    a = fma((double)rhs[i], A[i], a);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < RR; i += gridDim.x * blockDim.x) {
    double h = 1.0;
    for (int k = 0; k < N; k++) h *= S[(int64_t)k * RR + i];
    b += h;
  }
  __shared__ double ra[256], rb[256];
  ra[threadIdx.x] = a;
  rb[threadIdx.x] = b;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) {
      ra[threadIdx.x] += ra[threadIdx.x + st];
      rb[threadIdx.x] += rb[threadIdx.x + st];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = ra[0];
    part[2 * blockIdx.x + 1] = rb[0];
  }
}

__global__ void fitness_final_kernel(const double* __restrict__ part, int nparts, double normX2,
                                     double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double inner = 0.0, model = 0.0;
    for (int i = 0; i < nparts; i++) {
      inner += part[2 * i];
      model += part[2 * i + 1];
    }
    const double res2 = normX2 - 2.0 * inner + model;
    out[0] = 1.0 - sqrt(fmax(res2, 0.0)) / sqrt(normX2);
    out[1] = inner;
    out[2] = model;
  }
}

}  // namespace

// ---------------------------------------------------------------- host wrappers
cudaError_t setup_small_kernels() {
  const int g = (int)(kMaxRank * kMaxRank * sizeof(double));
  const int sv = (int)((kMaxRank * kMaxRank + kMaxRank) * sizeof(double));
  cudaError_t e = cudaFuncSetAttribute(gamma_chol_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, g);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(solve_rows_kernel<double, double>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, sv);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(solve_rows_kernel<float, float>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, sv);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(solve_rows_kernel<double, float>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, sv);
  return e;
}

void gamma_chol(const double* S, const double* W, int N, int n, int R, double* Lout, double* Z,
                bool useV, int* status, Launch L) {
  const size_t smem = (size_t)R * R * sizeof(double);
  gamma_chol_kernel<<<1, 512, smem, L.stream>>>(S, W, N, n, R, Lout, Z, useV ? 1 : 0, status);
  (*L.counter)++;
}

template <typename TR, typename T>
static void solve_launch(const TR* rhs, double* A, const double* Aref, double* dA, const double* Lf,
                         T* Ac, T* dAc, double* rownorm, int s, int R, int n, const int* status,
                         Launch L) {
  const size_t smem = (size_t)(R * R + R) * sizeof(double);
  const int rows_per_block = 4;
  const int blocks = (int)std::min<int64_t>(cdiv(s, rows_per_block), 152 * 2);
  solve_rows_kernel<TR, T><<<blocks, 32 * rows_per_block, smem, L.stream>>>(
      rhs, A, Aref, dA, Lf, Ac, dAc, rownorm, s, R, n, status);
  (*L.counter)++;
}

template <typename T>
void solve_rows(const T* rhs, double* A, const double* Aref, double* dA, const double* Lf, T* Ac,
                T* dAc, double* rownorm, int s, int R, int n, const int* status, Launch L) {
  solve_launch<T, T>(rhs, A, Aref, dA, Lf, Ac, dAc, rownorm, s, R, n, status, L);
}

template <typename T>
void solve_rows_v(const T* rhs, double* A, const double* Aref, double* dA, const double* Lf,
                  const double* Z, double* rhs2, T* Ac, T* dAc, double* rownorm, int s, int R,
                  int n, const int* status, Launch L) {
  const int64_t tot = (int64_t)s * R;
  vterm_kernel<T><<<(int)std::min<int64_t>(cdiv(tot, 256), 152 * 8), 256, 0, L.stream>>>(
      rhs, A, Z, rhs2, s, R);
  (*L.counter)++;
  solve_launch<double, T>(rhs2, A, Aref, dA, Lf, Ac, dAc, rownorm, s, R, n, status, L);
}

template <typename T>
void vterm(const T* rhs, const double* A, const double* Z, double* out, int s, int R, Launch L) {
  const int64_t tot = (int64_t)s * R;
  vterm_kernel<T><<<(int)std::min<int64_t>(cdiv(tot, 256), 152 * 8), 256, 0, L.stream>>>(
      rhs, A, Z, out, s, R);
  (*L.counter)++;
}

void gram_update(const double* A, const double* dA, double* S, double* W, bool withW, int s,
                 int R, const double* rownorm, double* scal, double* partials, Launch L) {
  const int nb = (R + 31) / 32;
  const int ntS = nb * (nb + 1) / 2;
  const int ntiles = withW ? ntS + nb * nb : ntS;
  int splits = std::max(1, std::min((2 * 152) / ntiles, (s + 31) / 32));
  const int chunk = (int)cdiv(cdiv(s, splits), 32) * 32;
  splits = (int)cdiv(s, chunk);
  gram_part_kernel<<<ntiles * splits, 256, 0, L.stream>>>(A, dA, s, R, nb, ntS, ntiles, chunk,
                                                          partials);
  gram_reduce_kernel<<<std::max(1, ntiles * 4), 256, 0, L.stream>>>(
      partials, R, nb, ntS, ntiles, splits, withW, S, W, rownorm, s, scal);
  (*L.counter) += 2;
}

template <typename T>
void fitness(const T* rhs, const double* A, const double* S, int N, int R, int s, double normX2,
             double* out, double* partials, Launch L) {
  const int blocks = 128;
  fitness_part_kernel<T><<<blocks, 256, 0, L.stream>>>(rhs, A, S, N, R, s, partials);
  fitness_final_kernel<<<1, 32, 0, L.stream>>>(partials, blocks, normX2, out);
  (*L.counter) += 2;
}

template void solve_rows<double>(const double*, double*, const double*, double*, const double*,
                                 double*, double*, double*, int, int, int, const int*, Launch);
template void solve_rows<float>(const float*, double*, const double*, double*, const double*,
                                float*, float*, double*, int, int, int, const int*, Launch);
template void solve_rows_v<double>(const double*, double*, const double*, double*, const double*,
                                   const double*, double*, double*, double*, double*, int, int,
                                   int, const int*, Launch);
template void solve_rows_v<float>(const float*, double*, const double*, double*, const double*,
                                  const double*, double*, float*, float*, double*, int, int, int,
                                  const int*, Launch);
template void vterm<double>(const double*, const double*, const double*, double*, int, int, Launch);
template void vterm<float>(const float*, const double*, const double*, double*, int, int, Launch);
template void fitness<double>(const double*, const double*, const double*, int, int, int, double,
                              double*, double*, Launch);
template void fitness<float>(const float*, const double*, const double*, int, int, int, double,
                             double*, double*, Launch);

}  // namespace cpals
