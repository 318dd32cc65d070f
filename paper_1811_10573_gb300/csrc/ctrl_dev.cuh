// Learned sweep-type controller on the device: its history of the run, its
// feature vector and the network's forward pass as device functions, so that
// the decision can be taken inside the device loop of Algorithm 3 (one warp,
// no host round trip).  The host loop of cpals_run_controlled keeps
// its own copy of the history and features in cpals.cu; the formulas are the
// same.  The forward pass is also the body of mlp_forward_kernel.
#pragma once

#include <cuda_runtime.h>

namespace cpals {

// actions (the network's classes)
enum CtrlAction { ACT_PP = 0, ACT_ALS = 1, ACT_REBUILD = 2 };

struct CtrlState {
  double maxlr[2];        // largest log10 ||dA||/||A|| of the last two sweeps
  double res[4];          // residual 1 - f of the last four sweeps (newest first; -1: none)
  int since_build;        // sweeps since the operators were built
  int pp_ready;           // operators built and only PP sweeps since
  int last;               // last action (-1: none)
  int pad;
};

__host__ __device__ inline void ctrl_state_start(CtrlState& h, double fitness) {
  h.maxlr[0] = h.maxlr[1] = 0.0;
  h.res[0] = 1.0 - fitness;
  h.res[1] = h.res[2] = h.res[3] = -1.0;
  h.since_build = 0;
  h.pp_ready = 0;
  h.last = -1;
  h.pad = 0;
}

// log10 ||dA^(n)|| / ||A^(n)|| of mode n (floored at 1e-12) from the scalars
// scal ([8 + 2n] ||dA^(n)||^2, [9 + 2n] ||A^(n)||^2)
__device__ inline double ctrl_mode_lr(const double* scal, int n) {
  const double d = sqrt(scal[8 + 2 * n]), a = sqrt(scal[9 + 2 * n]);
  return log10(fmax(d / fmax(a, 1e-300), 1e-12));
}

// after a sweep of kind `action` whose modes gave lr[n] = ctrl_mode_lr and
// the fitness the algorithm saw
__device__ inline void ctrl_push(CtrlState& h, const double* lr, int N, int action, double fitness) {
  double m = -12.0;
  for (int n = 0; n < N; n++) m = fmax(m, lr[n]);
  h.maxlr[1] = h.maxlr[0];
  h.maxlr[0] = m;
  for (int k = 3; k > 0; k--) h.res[k] = h.res[k - 1];
  h.res[0] = 1.0 - fitness;
  h.last = action;
  if (action == ACT_ALS) {
    h.pp_ready = 0;
    h.since_build = 0;
  } else if (action == ACT_REBUILD) {
    h.pp_ready = 1;
    h.since_build = 1;
  } else {
    h.since_build++;
  }
}

// feature i of the network's input (F = 20 values, all O(1)): per-mode
// log10 ||dA||/||A|| (padded to 8 modes), the largest one of the two
// previous sweeps, log10 of the last three residual decreases, sweeps since
// the operators were built, whether a PP sweep is possible, the last action
// (one-hot), log10 eps and log10 of the current residual.  One value per
// call, so that a warp forms all twenty at once (the float64 logarithms and
// square roots run on GB300's narrow FP64 pipe).
__device__ inline float ctrl_feature(const CtrlState& h, const double* lr, int N, double eps, int i) {
  if (i < 8) return i < N ? (float)(fmin(fmax(lr[i], -12.0), 2.0) / 4.0) : 0.f;
  if (i < 10) return (float)(h.maxlr[i - 8] / 4.0);
  if (i < 13) {
    const int k = i - 10;
    const bool have = h.res[k] >= 0 && h.res[k + 1] >= 0;
    const double dec = have ? fmax(h.res[k + 1] - h.res[k], 1e-16) : 1e-16;
    return (float)(log10(dec) / 8.0);
  }
  if (i == 13) return (float)(h.pp_ready ? fmin((double)h.since_build, 20.0) / 10.0 : 0.0);
  if (i == 14) return h.pp_ready ? 1.f : 0.f;
  if (i < 18) return h.last == i - 15 ? 1.f : 0.f;
  if (i == 18) return (float)(log10(fmax(eps, 1e-12)) / 2.0);
  return (float)(log10(fmax(h.res[0] >= 0 ? h.res[0] : 1.0, 1e-16)) / 8.0);
}

// probs = softmax(W2 relu(W1 x + b1) + b2); parameters W1[H][F], b1[H],
// W2[C][H], b2[C] with H = 32 hidden units and C = 3 classes
__device__ inline void mlp_probs(const float* __restrict__ params, int F, const float* x, float* probs) {
  constexpr int H = 32, C = 3;
  const float* W1 = params;
  const float* b1 = W1 + H * F;
  const float* W2 = b1 + H;
  const float* b2 = W2 + C * H;
  float h[H];
#pragma unroll 4
  for (int j = 0; j < H; j++) {
    float a = b1[j];
    for (int k = 0; k < F; k++) a = fmaf(W1[j * F + k], x[k], a);
    h[j] = fmaxf(a, 0.f);
  }
  float z[C], zmax = -3.4e38f;
  for (int c = 0; c < C; c++) {
    float a = b2[c];
#pragma unroll 4
    for (int j = 0; j < H; j++) a = fmaf(W2[c * H + j], h[j], a);
    z[c] = a;
    zmax = fmaxf(zmax, a);
  }
  float s = 0.f;
  for (int c = 0; c < C; c++) {
    z[c] = __expf(z[c] - zmax);
    s += z[c];
  }
  for (int c = 0; c < C; c++) probs[c] = z[c] / s;
}

// The same forward pass on one warp (all 32 lanes call it): lane j forms
// hidden unit j (the network has exactly 32) with mlp_probs' order of terms,
// and lane 0 forms the outputs in mlp_probs' order too, so the
// probabilities are bitwise those of mlp_probs.  x: the F inputs and hs:
// 32 floats of scratch, both in shared memory; probs is written by lane 0
// and visible to every lane on return.
template <int F>
__device__ inline void mlp_probs_warp(const float* __restrict__ params, const float* x, float* hs,
                                      float* probs) {
  constexpr int H = 32, C = 3;
  const int j = threadIdx.x & 31;
  const float* W1 = params;
  const float* b1 = W1 + H * F;
  const float* W2 = b1 + H;
  const float* b2 = W2 + C * H;
  float a = b1[j];
#pragma unroll
  for (int k = 0; k < F; k++) a = fmaf(W1[j * F + k], x[k], a);
  hs[j] = fmaxf(a, 0.f);
  __syncwarp();
  if (j == 0) {
    float z[C], zmax = -3.4e38f;
    for (int c = 0; c < C; c++) {
      float acc = b2[c];
#pragma unroll
      for (int q = 0; q < H; q++) acc = fmaf(W2[c * H + q], hs[q], acc);
      z[c] = acc;
      zmax = fmaxf(zmax, acc);
    }
    float sum = 0.f;
    for (int c = 0; c < C; c++) {
      z[c] = __expf(z[c] - zmax);
      sum += z[c];
    }
    for (int c = 0; c < C; c++) probs[c] = z[c] / sum;
  }
  __syncwarp();
}

}  // namespace cpals
