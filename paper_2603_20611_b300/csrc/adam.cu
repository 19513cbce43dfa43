// adam.cu -- the fit loop's parameter update (Sec. 5.1: Adam, the paper's
// initial learning rates decaying exponentially to a final ratio), sm_103a.
//
// One thread per Gaussian reads its 11 parameters, 11 gradients and 26 state
// floats and writes 11 parameters and 22 state floats back: ~340 bytes per
// Gaussian, an HBM-bound elementwise pass.  The state is laid out [26][n] so
// that every row is read and written coalesced; the per-step scalars (rates of
// the four groups at step t, bias corrections) are computed once on the host
// in double precision.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "gp_internal.h"

namespace gp {

namespace {

constexpr int kAdamRows = 26;  // m[11], v[11], raw log s[3], raw logit alpha[1]
constexpr int kAdamThreads = 256;

struct AdamStep {
  float lr[4];      // mu, scale, quat, alpha at this step
  float inv_bc1;    // 1 / (1 - b1^t)
  float inv_sbc2;   // 1 / sqrt(1 - b2^t)
  float b1, b2, eps;
  int act;          // log-scale / logit-alpha parameterisation
};

// One Adam update of parameter theta with gradient g; m and v in, updated.
__device__ __forceinline__ float adam_one(float theta, float g, float& m, float& v, const AdamStep& p, float lr) {
  m = fmaf(p.b1, m, (1.0f - p.b1) * g);
  v = fmaf(p.b2, v, (1.0f - p.b2) * g * g);
  return theta - lr * (m * p.inv_bc1) / fmaf(sqrtf(v), p.inv_sbc2, p.eps);
}

// Every load of a Gaussian first, then the updates, then every store: the 26
// state rows share one base pointer, so stores to one row would otherwise hold
// back the loads of the next.
__global__ void __launch_bounds__(kAdamThreads) k_adam(AdamStep p, int64_t n, float* __restrict__ mu,
                                                      float* __restrict__ scale, float* __restrict__ quat,
                                                      float* __restrict__ alpha, const float* __restrict__ d_mu,
                                                      const float* __restrict__ d_scale,
                                                      const float* __restrict__ d_quat,
                                                      const float* __restrict__ d_alpha, float* __restrict__ st) {
  const int64_t i = (int64_t)blockIdx.x * kAdamThreads + threadIdx.x;
  if (i >= n) return;
  // parameters and gradients in the order mu xyz, scale xyz, quat wxyz, alpha
  float th[11], g[11], m[11], v[11], raw[4];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    th[k] = mu[3 * i + k];
    g[k] = d_mu[3 * i + k];
    th[3 + k] = scale[3 * i + k];
    g[3 + k] = d_scale[3 * i + k];
  }
  const float4 q = reinterpret_cast<const float4*>(quat)[i];
  const float4 gq = reinterpret_cast<const float4*>(d_quat)[i];
  th[6] = q.x; th[7] = q.y; th[8] = q.z; th[9] = q.w;
  g[6] = gq.x; g[7] = gq.y; g[8] = gq.z; g[9] = gq.w;
  th[10] = alpha[i];
  g[10] = d_alpha[i];
#pragma unroll
  for (int k = 0; k < 11; ++k) {
    m[k] = st[(int64_t)k * n + i];          // rows 0..10
    v[k] = st[(int64_t)(11 + k) * n + i];   // rows 11..21
  }
  if (p.act) {
#pragma unroll
    for (int k = 0; k < 4; ++k) raw[k] = st[(int64_t)(22 + k) * n + i];  // raw log s xyz, raw logit alpha
  }
  // positions
#pragma unroll
  for (int k = 0; k < 3; ++k) th[k] = adam_one(th[k], g[k], m[k], v[k], p, p.lr[0]);
  // scales: raw log s (gradient through s = exp(raw)) or linear s
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (p.act) {
      raw[k] = adam_one(raw[k], g[3 + k] * th[3 + k], m[3 + k], v[3 + k], p, p.lr[1]);
      th[3 + k] = expf(raw[k]);
    } else {
      th[3 + k] = adam_one(th[3 + k], g[3 + k], m[3 + k], v[3 + k], p, p.lr[1]);
    }
  }
  // quaternion (normalised inside the renderer, optimised as it is)
#pragma unroll
  for (int k = 6; k < 10; ++k) th[k] = adam_one(th[k], g[k], m[k], v[k], p, p.lr[2]);
  // intensity: raw logit (gradient through a = sigmoid(raw)) or linear
  if (p.act) {
    const float a = th[10];
    raw[3] = adam_one(raw[3], g[10] * a * (1.0f - a), m[10], v[10], p, p.lr[3]);
    th[10] = 1.0f / (1.0f + expf(-raw[3]));
  } else {
    th[10] = adam_one(th[10], g[10], m[10], v[10], p, p.lr[3]);
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    mu[3 * i + k] = th[k];
    scale[3 * i + k] = th[3 + k];
  }
  reinterpret_cast<float4*>(quat)[i] = make_float4(th[6], th[7], th[8], th[9]);
  alpha[i] = th[10];
#pragma unroll
  for (int k = 0; k < 11; ++k) {
    st[(int64_t)k * n + i] = m[k];
    st[(int64_t)(11 + k) * n + i] = v[k];
  }
  if (p.act) {
#pragma unroll
    for (int k = 0; k < 4; ++k) st[(int64_t)(22 + k) * n + i] = raw[k];
  }
}

__global__ void __launch_bounds__(kAdamThreads) k_adam_init(int64_t n, const float* __restrict__ scale,
                                                           const float* __restrict__ alpha, int act,
                                                           float* __restrict__ st) {
  const int64_t i = (int64_t)blockIdx.x * kAdamThreads + threadIdx.x;
  if (i >= n) return;
#pragma unroll
  for (int r = 0; r < 22; ++r) st[r * n + i] = 0.0f;
  float* RAW = st + 22 * n;
  if (act) {
#pragma unroll
    for (int k = 0; k < 3; ++k) RAW[k * n + i] = logf(scale[3 * i + k]);
    const float a = fminf(fmaxf(alpha[i], 1e-6f), 1.0f - 1e-6f);
    RAW[3 * n + i] = logf(a) - log1pf(-a);
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) RAW[k * n + i] = 0.0f;
  }
}

bool cfg_ok(const gp_adam_cfg* c) {
  return c && c->lr_mu >= 0.f && c->lr_scale >= 0.f && c->lr_quat >= 0.f && c->lr_alpha >= 0.f &&
         isfinite(c->lr_mu) && isfinite(c->lr_scale) && isfinite(c->lr_quat) && isfinite(c->lr_alpha) &&
         c->mu_extent > 0.f && isfinite(c->mu_extent) && c->lr_final_ratio > 0.f && c->total_steps > 0 &&
         c->beta1 >= 0.f && c->beta1 < 1.f && c->beta2 >= 0.f && c->beta2 < 1.f && c->eps >= 0.f;
}

}  // namespace

}  // namespace gp

using namespace gp;

extern "C" {

gp_status gp_adam_default(gp_adam_cfg* cfg) {
  if (!cfg) return GP_ERR_ARG;
  cfg->lr_mu = 6e-4f;
  cfg->lr_scale = 2e-3f;
  cfg->lr_quat = 1e-3f;
  cfg->lr_alpha = 2e-2f;
  cfg->mu_extent = 1.0f;
  cfg->lr_final_ratio = 0.1f;
  cfg->total_steps = 30000;
  cfg->beta1 = 0.9f;
  cfg->beta2 = 0.999f;
  cfg->eps = 1e-15f;
  cfg->log_scale_logit_alpha = 1;
  return GP_OK;
}

int64_t gp_adam_state_floats(int64_t n) { return n > 0 ? (int64_t)kAdamRows * n : 0; }

gp_status gp_adam_init(gp_ctx* ctx, const gp_adam_cfg* cfg, int64_t n, const float* scale, const float* alpha,
                       float* state, void* stream) {
  if (!ctx) return GP_ERR_ARG;
  Ctx* c = &ctx->impl;
  if (!cfg_ok(cfg) || n < 0) return set_err(c, GP_ERR_ARG, "bad Adam configuration or size");
  if (n == 0) return GP_OK;
  if (!scale || !alpha || !state) return set_err(c, GP_ERR_ARG, "NULL pointer");
  if (cudaSetDevice(c->device) != cudaSuccess) return cuda_err(c, cudaGetLastError(), "cudaSetDevice");
  k_adam_init<<<(unsigned)((n + kAdamThreads - 1) / kAdamThreads), kAdamThreads, 0, (cudaStream_t)stream>>>(
      n, scale, alpha, cfg->log_scale_logit_alpha ? 1 : 0, state);
  note_launch();
  return cuda_err(c, cudaGetLastError(), "adam init");
}

gp_status gp_adam_step(gp_ctx* ctx, const gp_adam_cfg* cfg, int64_t t, int64_t n, float* mu, float* scale,
                       float* quat, float* alpha, const float* d_mu, const float* d_scale, const float* d_quat,
                       const float* d_alpha, float* state, void* stream) {
  if (!ctx) return GP_ERR_ARG;
  Ctx* c = &ctx->impl;
  if (!cfg_ok(cfg) || n < 0 || t < 1) return set_err(c, GP_ERR_ARG, "bad Adam configuration, size or step");
  if (n == 0) return GP_OK;
  if (!mu || !scale || !quat || !alpha || !d_mu || !d_scale || !d_quat || !d_alpha || !state)
    return set_err(c, GP_ERR_ARG, "NULL pointer");
  if (((uintptr_t)quat & 15u) || ((uintptr_t)d_quat & 15u))
    return set_err(c, GP_ERR_ARG, "quat and d_quat must be 16-byte aligned");
  if (cudaSetDevice(c->device) != cudaSuccess) return cuda_err(c, cudaGetLastError(), "cudaSetDevice");
  const double k = (double)std::min<int64_t>(t - 1, cfg->total_steps);
  const double decay = pow((double)cfg->lr_final_ratio, k / (double)cfg->total_steps);
  AdamStep p;
  p.lr[0] = (float)((double)cfg->lr_mu * cfg->mu_extent * decay);
  p.lr[1] = (float)((double)cfg->lr_scale * decay);
  p.lr[2] = (float)((double)cfg->lr_quat * decay);
  p.lr[3] = (float)((double)cfg->lr_alpha * decay);
  p.inv_bc1 = (float)(1.0 / (1.0 - pow((double)cfg->beta1, (double)t)));
  p.inv_sbc2 = (float)(1.0 / sqrt(1.0 - pow((double)cfg->beta2, (double)t)));
  p.b1 = cfg->beta1;
  p.b2 = cfg->beta2;
  p.eps = cfg->eps;
  p.act = cfg->log_scale_logit_alpha ? 1 : 0;
  cudaStream_t st = (cudaStream_t)stream;
  PhaseTimer timer(c, GP_PHASE_OPT, st);
  k_adam<<<(unsigned)((n + kAdamThreads - 1) / kAdamThreads), kAdamThreads, 0, st>>>(
      p, n, mu, scale, quat, alpha, d_mu, d_scale, d_quat, d_alpha, state);
  note_launch();
  return cuda_err(c, cudaGetLastError(), "adam step");
}

}  // extern "C"
