// Learned sweep-type controller: a two-layer perceptron (F inputs, 32 hidden
// ReLU units, 3 outputs with softmax) that picks the next sweep of PP-CP-ALS
// among a PP approximated sweep, an exact ALS sweep and an operator rebuild
// followed by a PP sweep (the choices Algorithm 3 makes with its eps test;
// Sec. 6 of the paper invites other switching schemes).  Inference and
// training are these kernels; the run loop and the feature vector live in
// cpals.cu.
//
// Parameter layout (float): W1[H][F], b1[H], W2[C][H], b2[C].
// Training is full-batch Adam on a weighted cross-entropy: per epoch one
// kernel runs every sample forward and backward (one thread per sample) and
// stores its hidden activations and output/hidden deltas, a second kernel
// gives each parameter its gradient as a sum over the samples in index order
// (deterministic) and applies the Adam step.
#include "ctrl_dev.cuh"
#include "internal.h"

namespace cpals {

namespace {

constexpr int H = kCtrlHidden;
constexpr int C = kCtrlClasses;
static_assert(H == 32 && C == 3 && kCtrlFeatures == 20, "mlp_probs and ctrl_feature are written for 20-32-3");

struct Params {
  const float* W1;
  const float* b1;
  const float* W2;
  const float* b2;
};

__device__ __forceinline__ Params view(const float* p, int F) {
  return {p, p + H * F, p + H * F + H, p + H * F + H + C * H};
}

// out[i][c] = softmax(W2 relu(W1 x_i + b1) + b2) (the device loop's decide
// kernel takes the same forward pass, mlp_probs)
__global__ void mlp_forward_kernel(const float* __restrict__ params, int F,
                                   const float* __restrict__ X, int n, float* __restrict__ probs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  mlp_probs(params, F, X + (size_t)i * F, probs + (size_t)i * C);
}

// per sample: hidden activations, output delta w_i (p - onehot(y_i)) and
// hidden delta (W2^T dz) * [h > 0]; loss_i = -w_i log p_y
__global__ void mlp_backprop_kernel(const float* __restrict__ params, int F,
                                    const float* __restrict__ X, const int* __restrict__ y,
                                    const float* __restrict__ w, int n, float* __restrict__ hs,
                                    float* __restrict__ dz, float* __restrict__ dh,
                                    float* __restrict__ loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Params P = view(params, F);
  const float* x = X + (size_t)i * F;
  float h[H];
#pragma unroll 4
  for (int j = 0; j < H; j++) {
    float a = P.b1[j];
    for (int k = 0; k < F; k++) a = fmaf(P.W1[j * F + k], x[k], a);
    h[j] = fmaxf(a, 0.f);
    hs[(size_t)i * H + j] = h[j];
  }
  float z[C], zmax = -3.4e38f;
  for (int c = 0; c < C; c++) {
    float a = P.b2[c];
#pragma unroll 4
    for (int j = 0; j < H; j++) a = fmaf(P.W2[c * H + j], h[j], a);
    z[c] = a;
    zmax = fmaxf(zmax, a);
  }
  float s = 0.f;
  for (int c = 0; c < C; c++) {
    z[c] = __expf(z[c] - zmax);
    s += z[c];
  }
  const float wi = w[i];
  const int yi = y[i];
  float d[C];
  for (int c = 0; c < C; c++) {
    const float p = z[c] / s;
    d[c] = wi * (p - (c == yi ? 1.f : 0.f));
    dz[(size_t)i * C + c] = d[c];
  }
  loss[i] = -wi * __logf(fmaxf(z[yi] / s, 1e-30f));
  for (int j = 0; j < H; j++) {
    float a = 0.f;
    for (int c = 0; c < C; c++) a = fmaf(P.W2[c * H + j], d[c], a);
    dh[(size_t)i * H + j] = h[j] > 0.f ? a : 0.f;
  }
}

// parameter q: gradient = (1/W) sum over samples in index order, plus decay
// on the weights; then Adam (bias-corrected) with step t (1-based)
__global__ void mlp_adam_kernel(float* __restrict__ params, float* __restrict__ m,
                                float* __restrict__ v, int F, const float* __restrict__ X,
                                const float* __restrict__ hs, const float* __restrict__ dz,
                                const float* __restrict__ dh, int n, float inv_w, float lr,
                                float decay, int t) {
  const int nW1 = H * F, nb1 = H, nW2 = C * H, nb2 = C;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nW1 + nb1 + nW2 + nb2) return;
  float g = 0.f;
  bool weight = false;
  if (q < nW1) {
    const int j = q / F, k = q % F;
    for (int i = 0; i < n; i++) g = fmaf(dh[(size_t)i * H + j], X[(size_t)i * F + k], g);
    weight = true;
  } else if (q < nW1 + nb1) {
    const int j = q - nW1;
    for (int i = 0; i < n; i++) g += dh[(size_t)i * H + j];
  } else if (q < nW1 + nb1 + nW2) {
    const int r = q - nW1 - nb1, c = r / H, j = r % H;
    for (int i = 0; i < n; i++) g = fmaf(dz[(size_t)i * C + c], hs[(size_t)i * H + j], g);
    weight = true;
  } else {
    const int c = q - nW1 - nb1 - nW2;
    for (int i = 0; i < n; i++) g += dz[(size_t)i * C + c];
  }
  g *= inv_w;
  if (weight) g += decay * params[q];
  const float b1 = 0.9f, b2 = 0.999f;
  const float mq = b1 * m[q] + (1.f - b1) * g;
  const float vq = b2 * v[q] + (1.f - b2) * g * g;
  m[q] = mq;
  v[q] = vq;
  const float mh = mq / (1.f - powf(b1, (float)t));
  const float vh = vq / (1.f - powf(b2, (float)t));
  params[q] -= lr * mh / (sqrtf(vh) + 1e-8f);
}

}  // namespace

int ctrl_param_count(int F) { return H * F + H + C * H + C; }

void mlp_forward(const float* params, int F, const float* X, int n, float* probs, Launch L) {
  mlp_forward_kernel<<<(n + 127) / 128, 128, 0, L.stream>>>(params, F, X, n, probs);
  (*L.counter)++;
}

void mlp_train_epoch(float* params, float* m, float* v, int F, const float* X, const int* y,
                     const float* w, int n, float inv_w, float lr, float decay, int t, float* hs,
                     float* dz, float* dh, float* loss, Launch L) {
  mlp_backprop_kernel<<<(n + 127) / 128, 128, 0, L.stream>>>(params, F, X, y, w, n, hs, dz, dh, loss);
  const int np = ctrl_param_count(F);
  mlp_adam_kernel<<<(np + 127) / 128, 128, 0, L.stream>>>(params, m, v, F, X, hs, dz, dh, n, inv_w,
                                                          lr, decay, t);
  (*L.counter) += 2;
}

}  // namespace cpals
