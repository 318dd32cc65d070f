// Internal declarations shared by the translation units of libcpals.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>

namespace cpals {

// Where a launch goes and the counter of kernels launched.
struct Launch {
  cudaStream_t stream;
  int64_t* counter;
};

constexpr int kMaxModes = 8;
constexpr int kMaxRank = 128;

// ---------------------------------------------------------------- contractions
// First-level contraction of the tensor with a factor (or Khatri-Rao product)
// B (K x R, r fastest), Sec. 2.5:
//   kmajor:  out[m][r]    = sum_k X[m*K + k]          * B[k][r]   (batch must be 1)
//   !kmajor: out[b][m][r] = sum_k X[(b*K + k)*M + m]  * B[k][r]
// splits > 1 splits K; partials (splits*batch*M*R values) then holds the
// partial sums and a deterministic reduction writes out.  part_cap > 0 (the
// values partials holds) lets a float64 K-major launch of one batch with
// splits == 1 split K for the rows of its last, partial wave.
template <typename TX, typename T>
void gemm_simt(const TX* X, const T* B, T* out, T* partials, int64_t batch, int64_t K, int64_t M,
               int R, bool kmajor, int splits, Launch L, int64_t part_cap = 0);

// K splits for a float64 gemm_simt: with R > 32 (64-row exact-column tiles)
// the grid is about four waves of resident CTAs when the output alone does
// not fill the GPU (1 when it does); otherwise K is split until every SM has
// a CTA (at least 16 k per split).  0 for other types.
int gemm_simt_wave_splits(int64_t batch, int64_t K, int64_t M, int R, bool kmajor, size_t esz,
                          int64_t cap);

// K splits for gemm_simt so that its grid has at least min_blocks CTAs
// (at least 64 k per split; splits * batch * M * R must fit in cap values).
int gemm_simt_splits(int64_t batch, int64_t K, int64_t M, int R, bool kmajor, int64_t cap,
                     int min_blocks);

// out[i] = sum_z part[z*n + i], deterministic order.
template <typename T>
void reduce_splits(const T* part, T* out, int64_t n, int splits, Launch L);

// Multi-TTV (lower levels of the trees): out[o][q][r] = sum_x in[o][x][q][r] * A[x][r].
template <typename T>
void ttv(const T* in, const T* A, T* out, int64_t outer, int sw, int64_t inner, int R, Launch L);

// One first-order term of Eq. 3: out[y][r] += sum_x op[y*ystride + x*xstride + r] * dA[x][r].
template <typename T>
struct PPTerm {
  const T* op;
  const T* dA;
  int64_t xstride;
  int64_t ystride;
  int sx;
};
// out[y][r] = Mp[y][r] + sum over terms (Eq. 3, first two terms).
template <typename T>
void pp_correct(const T* Mp, const PPTerm<T>* terms, int nterms, T* out, int sy, int R, Launch L);

// Row-major Khatri-Rao product of nm factors (last factor fastest): out is prod(dims) x R.
template <typename T>
void khatri_rao(const T* const* A, const int64_t* dims, int nm, int R, T* out, Launch L);

// Same product written transposed, zero-padded and split into two bf16 planes
// for the tensor cores: outT[0][r][k] = hi = bf16(v), outT[1][r][k] =
// bf16(v - hi), r < Rpad, k < Kstride (k >= K and r >= R are zero).
void khatri_rao_bf16_t(const float* const* A, const int64_t* dims, int nm, int R, int Rpad,
                       int64_t Kstride, __nv_bfloat16* outT, Launch L);

// Element conversions.
template <typename TS, typename TD>
void convert(const TS* src, TD* dst, int64_t n, Launch L);

// sum of squares of n values, accumulated in float64 (deterministic two-pass).
template <typename TX>
void sumsq(const TX* x, int64_t n, double* partials, double* out, Launch L);

// ---------------------------------------------------------------- float64 small kernels
// Gamma^(n) = *_{k != n} S^(k) (Algorithm 1), its Cholesky factor L (R x R in
// Lout), and (useV) Z = sum_{i<j; i,j != n} W_i * W_j * (*_{k not in {i,j,n}}
// S_k) so that sum_{i<j} V^(n,i,j) = A^(n) Z (Eq. 3).  A Gamma that is not
// positive definite leaves Gamma^dagger in Lout instead, with status[0] bit
// 16 + n; status[0] |= 1<<n if Gamma is not finite.
void gamma_chol(const double* S, const double* W, int N, int n, int R, double* Lout, double* Z,
                bool useV, int* status, Launch L);

// Row-wise solve A_new = rhs Gamma^{-1} with the factor L (or Gamma^dagger); writes A (in place),
// dA = A_new - (Aref ? Aref : A_old), compute-precision copies Ac, dAc and per-row
// ||dA||^2, ||A_new||^2 into rownorm (2*s values).  Rows are left unchanged if
// the factorisation failed for this mode (status bit set).  lam is the update
// step size (Sec. 5.1): A_new = (1 - lam) A_old + lam rhs Gamma^{-1}.
template <typename T>
void solve_rows(const T* rhs, double* A, const double* Aref, double* dA, const double* Lf, T* Ac,
                T* dAc, double* rownorm, int s, int R, int n, double lam, const int* status,
                Launch L);
// Same with the second-order PP terms: rhs2 = rhs + A_old Z (compute precision,
// s*R scratch values) is formed first from the compute copy Ac of A_old.
template <typename T>
void solve_rows_v(const T* rhs, double* A, const double* Aref, double* dA, const double* Lf,
                  const double* Z, T* rhs2, T* Ac, T* dAc, double* rownorm, int s, int R, int n,
                  double lam, const int* status, Launch L);
// out[y][r] = rhs[y][r] + sum_k A[y][k] Z[k][r] in the compute precision.
template <typename T>
void vterm(const T* rhs, const T* A, const double* Z, T* out, int s, int R, Launch L);
// The same with a float Z (the double-float path's second-order terms).
void vterm_fz(const float* rhs, const float* A, const float* Z, float* out, int s, int R, Launch L);
// Raise the dynamic shared-memory limits of the float64 kernels (call once per device).
cudaError_t setup_small_kernels();

// S = A^T A in float64 and (withW) W = Ac^T dAc in the compute precision T;
// also reduces rownorm into scal[0] = ||dA||^2, scal[1] = ||A||^2.
// partials: ceil(s/32) * 26 * 1024 float64 scratch; tickets: 64 ints, zero
// before the first launch (each launch leaves them zero).
template <typename T>
void gram_update(const double* A, const T* Ac, const T* dAc, double* S, double* W, bool withW,
                 int s, int R, const double* rownorm, double* scal, double* partials, int* tickets,
                 Launch L);

// Fitness from the last mode's right-hand side (Sec. 5), with ||X||^2 read
// from device memory at run time (normX2):
// inner = sum rhs*A, model = sum_{r,r'} prod_k S_k, out[0] = fitness, out[1] = inner,
// out[2] = model.  partials: workspace (>= 2*256 doubles); ticket: one zeroed
// int (the last block resets it), shared only by launches on one stream.
template <typename T>
void fitness(const T* rhs, const double* A, const double* S, int N, int R, int s,
             const double* normX2, double* out, double* partials, int* ticket, Launch L);

// ---------------------------------------------------------------- double-float (FP32/mixed modes)
// The same normal-equation steps in double-float arithmetic (hi + lo floats)
// on the float32 pipes.  Factors are carried as Ahi (= the float compute copy)
// and Alo; Grams as S (float64), Shi, Slo; W and Z in float.
cudaError_t setup_df_kernels();
void split_df(const double* A, float* hi, float* lo, int64_t n, Launch L);
void gram_df(const float* Ahi, const float* Alo, const float* Aw, const float* dAw, double* S,
             float* Shi, float* Slo, float* W, bool withW, int s, int R, const float2* rownorm,
             double* scal, const float* ShiAll, const float* SloAll, int N, int n, int nn,
             float2* Gpk, Launch L);
// gram_df with nn >= 0 also writes Gamma^(nn) (the next mode's) packed by
// columns into Gpk; chol_df: Gamma^(n) (from Gpk when not null, else from the
// Grams) = L L^T and Winv = L^-1 (row stride R|1, zero upper triangle);
// solve_df: a = Winv^T Winv b per row, blended with the old row when the
// update step size lam != 1 (Sec. 5.1).
void chol_df(const float* Shi, const float* Slo, const float* W, const float2* Gpk, int N, int n,
             int R, float2* Winv, float* Z, bool useV, int* status, Launch L);
void solve_df(const float* rhs, double* A, float* Ahi, float* Alo, const float* Arefhi,
              const float* Areflo, double* dA, float* dAc, const float2* Winv, const float* Z,
              float2* rownorm, int s, int R, int n, double lam, const int* status, Launch L);

// ---------------------------------------------------------------- learned controller
// two-layer perceptron: kCtrlFeatures inputs, kCtrlHidden ReLU units,
// kCtrlClasses outputs (PP sweep, ALS sweep, rebuild + PP sweep)
constexpr int kCtrlFeatures = 20;
constexpr int kCtrlHidden = 32;
constexpr int kCtrlClasses = 3;
int ctrl_param_count(int F);
void mlp_forward(const float* params, int F, const float* X, int n, float* probs, Launch L);
void mlp_train_epoch(float* params, float* m, float* v, int F, const float* X, const int* y,
                     const float* w, int n, float inv_w, float lr, float decay, int t, float* hs,
                     float* dz, float* dh, float* loss, Launch L);

// ---------------------------------------------------------------- tcgen05 (sm_103a)
// bf16 tensor-core first-level contraction, fp32 accumulate in TMEM, TMA-fed:
//   kmajor:  out[m][r]    = sum_k Xb[m*K + k]         * Bt[r][k]
//   !kmajor: out[b][m][r] = sum_k Xb[(b*K + k)*M + m] * Bt[r][k]
// Bt holds two planes (hi, lo) of Rpad (multiple of 16) rows x Kstride bf16
// (zero padded); the product uses hi + lo.
// splits > 1: fp32 partials + deterministic reduction into out.
// sched: two zeroed ints that launches on one stream may share (units are
// handed out dynamically and the counter is reset by the kernel); null gives
// a static round-robin assignment (safe for concurrent launches).
// wait_limit: bound of the kernel's waits on work in SM clock cycles (0 = the
// default, about 2 s); on expiry the kernel writes a nonzero code to *err_flag,
// lets what it already issued land and returns.
// Returns false if the shape is not supported (alignment), so the caller can
// report CPALS_E_UNSUPPORTED.
bool umma_supported(int64_t K, int64_t M, bool kmajor, int R);
// Raise the dynamic shared-memory limit of the tensor-core kernels (once per device).
cudaError_t setup_umma_kernels();
cudaError_t umma_gemm_bf16(const __nv_bfloat16* Xb, const __nv_bfloat16* Bt, float* out,
                           float* partials, int64_t batch, int64_t K, int64_t M, int R, int Rpad,
                           int64_t Kstride, bool kmajor, int splits, int* err_flag, int* sched,
                           Launch L, uint64_t wait_limit = 0);

}  // namespace cpals
