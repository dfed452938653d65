// Learned rank / skeleton proposer: box features, a 128-128-128 ReLU MLP with FP16
// weights and FP32 accumulation, its loss, backward pass and Adam optimiser -- the
// network's training and inference kernels.  The proposer is an addition to the paper's
// method (which chooses ranks by the ID tolerance alone, Sec. 4.1): its rank proposals
// size the randomized sketch of each column ID, and every sketched ID is accepted only
// after the residual check of idcheck.cu, else redone as the plain ID.
//
// Features of a box with nodes [begin, begin + L), centre c, radius rho (0 read as 1):
//   for j = 0..31, node q_j = begin + ((2j + 1) L) / 64 (integer division):
//     f[3j] = (x_q - cx) / rho, f[3j + 1] = (y_q - cy) / rho, f[3j + 2] = kappa_q rho;
//   f[96] = 2 rho k0 / 32, f[97] = 2 rho k1 / 32, f[98] = -log10(tol) / 10,
//   f[99] = height / 8, f[100] = log2(1 + n_act0) / 8, f[101] = log2(1 + n_act1) / 8,
//   f[102] = log2(1 + m_near) / 8, f[103] = nproxy / 256, f[104..127] = 0.
// Targets of a box (from a plain ID): y[h] = log2(1 + rank_h) / 8 and, per position
// j = ((q - begin) 32) / L of its active nodes q, the fraction that are skeleton nodes.
//
// Loss over B boxes: (1/B) sum (o_h - y_h)^2 + (0.1 / 64B) sum mask * BCE(sigmoid(o), t).
#include <cuda_fp16.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"

namespace symhss {

namespace {

constexpr int kW = kMlpWidth;
static_assert(kMlpParams == SYMHSS_MLP_PARAMS && kMlpWidth == SYMHSS_MLP_WIDTH, "packed parameter layout");
constexpr int kTB = 16;          // samples per block of the dense kernels
constexpr float kLam = 0.1f;

__global__ void __launch_bounds__(kW) box_features_kernel(const PointTable t, const FeatJob* jobs, float* out) {
  const FeatJob jb = jobs[blockIdx.x];
  const int f = threadIdx.x;
  const double r = jb.rho > 0.0 ? jb.rho : 1.0;
  double v = 0.0;
  if (f < 96) {
    const int j = f / 3;
    const int q = jb.begin + ((2 * j + 1) * jb.len) / 64;
    const int c = f - 3 * j;
    v = c == 0 ? (t.x[q] - jb.cx) / r : (c == 1 ? (t.y[q] - jb.cy) / r : t.kappa[q] * r);
  } else if (f == 96) v = 2.0 * jb.rho * jb.k0 / 32.0;
  else if (f == 97) v = 2.0 * jb.rho * jb.k1 / 32.0;
  else if (f == 98) v = jb.tol > 0.0 ? -log10(jb.tol) / 10.0 : 3.2;
  else if (f == 99) v = jb.height / 8.0;
  else if (f == 100) v = log2(1.0 + jb.n0) / 8.0;
  else if (f == 101) v = log2(1.0 + jb.n1) / 8.0;
  else if (f == 102) v = log2(1.0 + jb.m_near) / 8.0;
  else if (f == 103) v = jb.nproxy / 256.0;
  out[(long long)blockIdx.x * kW + f] = (float)v;
}

// Y[b, o] = act(sum_i W[o, i] X[b, i] + bias[o]); W, bias: one layer of the FP16 parameters.
__global__ void __launch_bounds__(kW) dense_fwd_kernel(const __half* Wb, const float* X, float* Y, int B, int relu) {
  __shared__ __half wt[kW * kW];  // wt[i * kW + o] = W[o, i]
  __shared__ float xs[kTB][kW];
  const int o = threadIdx.x;
  for (int e = o; e < kW * kW; e += kW) wt[(e % kW) * kW + e / kW] = Wb[e];
  const int b0 = blockIdx.x * kTB;
  for (int e = o; e < kTB * kW; e += kW) {
    const int s = e / kW, i = e % kW;
    xs[s][i] = b0 + s < B ? X[(long long)(b0 + s) * kW + i] : 0.0f;
  }
  __syncthreads();
  const float bias = __half2float(Wb[kW * kW + o]);
  float acc[kTB];
#pragma unroll
  for (int s = 0; s < kTB; ++s) acc[s] = bias;
  for (int i = 0; i < kW; ++i) {
    const float w = __half2float(wt[i * kW + o]);
#pragma unroll
    for (int s = 0; s < kTB; ++s) acc[s] = fmaf(w, xs[s][i], acc[s]);
  }
#pragma unroll
  for (int s = 0; s < kTB; ++s)
    if (b0 + s < B) Y[(long long)(b0 + s) * kW + o] = relu ? fmaxf(acc[s], 0.0f) : acc[s];
}

// dZ_low[b, i] = (sum_o W[o, i] dZ[b, o]) * (H_low[b, i] > 0)
__global__ void __launch_bounds__(kW) dense_bwd_input_kernel(const __half* Wb, const float* dZ, const float* Hl,
                                                             float* dZl, int B) {
  __shared__ __half w[kW * kW];
  __shared__ float ds[kTB][kW];
  const int i = threadIdx.x;
  for (int e = i; e < kW * kW; e += kW) w[e] = Wb[e];
  const int b0 = blockIdx.x * kTB;
  for (int e = i; e < kTB * kW; e += kW) {
    const int s = e / kW, o = e % kW;
    ds[s][o] = b0 + s < B ? dZ[(long long)(b0 + s) * kW + o] : 0.0f;
  }
  __syncthreads();
  float acc[kTB];
#pragma unroll
  for (int s = 0; s < kTB; ++s) acc[s] = 0.0f;
  for (int o = 0; o < kW; ++o) {
    const float wv = __half2float(w[o * kW + i]);
#pragma unroll
    for (int s = 0; s < kTB; ++s) acc[s] = fmaf(wv, ds[s][o], acc[s]);
  }
#pragma unroll
  for (int s = 0; s < kTB; ++s) {
    if (b0 + s >= B) continue;
    const long long k = (long long)(b0 + s) * kW + i;
    dZl[k] = Hl[k] > 0.0f ? acc[s] : 0.0f;
  }
}

// gW[o, i] = sum_b dZ[b, o] X[b, i] over 32 x 32 tiles (block 32 x 8, four rows per thread);
// gb[o] = sum_b dZ[b, o] by the blocks of the first column tile.
__global__ void __launch_bounds__(256) dense_bwd_weight_kernel(const float* dZ, const float* X, float* g, int B) {
  __shared__ float zs[32][33], xs[32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int o0 = blockIdx.y * 32, i0 = blockIdx.x * 32;
  float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  float bacc = 0.0f;
  for (int b0 = 0; b0 < B; b0 += 32) {
    for (int r = ty; r < 32; r += 8) {
      const int b = b0 + r;
      zs[r][tx] = b < B ? dZ[(long long)b * kW + o0 + tx] : 0.0f;
      xs[r][tx] = b < B ? X[(long long)b * kW + i0 + tx] : 0.0f;
    }
    __syncthreads();
    for (int r = 0; r < 32; ++r) {
      const float xv = xs[r][tx];
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[k] = fmaf(zs[r][ty + 8 * k], xv, acc[k]);
    }
    if (ty == 0 && blockIdx.x == 0)
      for (int r = 0; r < 32; ++r) bacc += zs[r][tx];
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) g[(long long)(o0 + ty + 8 * k) * kW + i0 + tx] = acc[k];
  if (ty == 0 && blockIdx.x == 0) g[kW * kW + o0 + tx] = bacc;
}

// dO and the loss (accumulated in FP64) from the outputs O and the targets.
__global__ void __launch_bounds__(kW) loss_kernel(const float* O, const float* yr, const float* ys, const float* mask,
                                                  float* dO, double* loss, int B) {
  __shared__ double part[kW / 32];
  const int b = blockIdx.x, o = threadIdx.x;
  const float z = O[(long long)b * kW + o];
  float d = 0.0f;
  double l = 0.0;
  if (o < 2) {
    const float r = z - yr[b * 2 + o];
    d = 2.0f * r / (float)B;
    l = (double)r * r / B;
  } else if (o < kMlpOutUsed) {
    const int j = o - 2;
    const float t = ys[(long long)b * 64 + j], mk = mask[(long long)b * 64 + j];
    const float p = 1.0f / (1.0f + expf(-z));
    const float c = kLam / (64.0f * (float)B);
    d = c * mk * (p - t);
    // BCE(sigmoid(z), t) = max(z, 0) - z t + log(1 + exp(-|z|))
    const double zd = z;
    l = (double)c * mk * (fmax(zd, 0.0) - zd * t + log1p(exp(-fabs(zd))));
  }
  dO[(long long)b * kW + o] = d;
  l = warp_sum(l);
  if ((o & 31) == 0) part[o >> 5] = l;
  __syncthreads();
  if (o == 0) {
    double sacc = 0.0;
    for (int w = 0; w < kW / 32; ++w) sacc += part[w];
    atomicAdd(loss, sacc);
  }
}

__global__ void adam_kernel(float* w, float* m, float* v, const float* g, __half* w16, int n, float lr, float c1,
                            float c2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float gk = g[k];
  const float mk = 0.9f * m[k] + 0.1f * gk;
  const float vk = 0.999f * v[k] + 0.001f * gk * gk;
  m[k] = mk;
  v[k] = vk;
  const float wk = w[k] - lr * (mk / c1) / (sqrtf(vk / c2) + 1e-8f);
  w[k] = wk;
  w16[k] = __float2half_rn(wk);
}

__global__ void to_half_kernel(const float* w, __half* w16, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) w16[k] = __float2half_rn(w[k]);
}

}  // namespace

cudaError_t launch_box_features(const PointTable& t, const FeatJob* jobs, int njobs, float* out, cudaStream_t s) {
  if (njobs <= 0) return cudaSuccess;
  box_features_kernel<<<njobs, kW, 0, s>>>(t, jobs, out);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace symhss

using namespace symhss;

struct symhss_mlp_s {
  int max_batch = 0;
  float *master = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
  __half* w16 = nullptr;
  float* act = nullptr;   // H1, H2, O, dO, dZ2, dZ1: max_batch x 128 each
  double* loss = nullptr;
  long long step = 0;
  ~symhss_mlp_s() {
    for (void* p : {(void*)master, (void*)m, (void*)v, (void*)grad, (void*)w16, (void*)act, (void*)loss})
      if (p) cudaFree(p);
  }
};

namespace symhss {

namespace {

int to_status(cudaError_t e) { return e == cudaErrorMemoryAllocation ? SYMHSS_ERR_NOMEM : SYMHSS_ERR_CUDA; }

float* act_buf(symhss_mlp_s* n, int k) { return n->act + (size_t)k * n->max_batch * kW; }

// Forward of B <= max_batch samples; outputs in act buffer 2 (O), hidden layers in 0, 1.
cudaError_t forward_chunk(symhss_mlp_s* n, const float* x, int B, cudaStream_t s) {
  const int grid = (B + kTB - 1) / kTB;
  const __half* w = n->w16;
  dense_fwd_kernel<<<grid, kW, 0, s>>>(w, x, act_buf(n, 0), B, 1);
  dense_fwd_kernel<<<grid, kW, 0, s>>>(w + kMlpLayerParams, act_buf(n, 0), act_buf(n, 1), B, 1);
  dense_fwd_kernel<<<grid, kW, 0, s>>>(w + 2 * kMlpLayerParams, act_buf(n, 1), act_buf(n, 2), B, 0);
  count_launches(3);
  return cudaGetLastError();
}

// Loss and gradient (into n->grad) of one batch of B <= max_batch samples.
cudaError_t loss_grad_chunk(symhss_mlp_s* n, const float* x, const float* yr, const float* ys, const float* mask,
                            int B, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(n->loss, 0, sizeof(double), s);
  if (e != cudaSuccess) return e;
  e = forward_chunk(n, x, B, s);
  if (e != cudaSuccess) return e;
  float *H1 = act_buf(n, 0), *H2 = act_buf(n, 1), *O = act_buf(n, 2), *dO = act_buf(n, 3);
  float *dZ2 = act_buf(n, 4), *dZ1 = act_buf(n, 5);
  loss_kernel<<<B, kW, 0, s>>>(O, yr, ys, mask, dO, n->loss, B);
  const int grid = (B + kTB - 1) / kTB;
  const __half* w = n->w16;
  const dim3 wg(kW / 32, kW / 32), wb(32, 8);
  float* g = n->grad;
  dense_bwd_weight_kernel<<<wg, wb, 0, s>>>(dO, H2, g + 2 * kMlpLayerParams, B);
  dense_bwd_input_kernel<<<grid, kW, 0, s>>>(w + 2 * kMlpLayerParams, dO, H2, dZ2, B);
  dense_bwd_weight_kernel<<<wg, wb, 0, s>>>(dZ2, H1, g + kMlpLayerParams, B);
  dense_bwd_input_kernel<<<grid, kW, 0, s>>>(w + kMlpLayerParams, dZ2, H1, dZ1, B);
  dense_bwd_weight_kernel<<<wg, wb, 0, s>>>(dZ1, x, g, B);
  count_launches(6);
  return cudaGetLastError();
}

}  // namespace

// Forward pass used by the solver (features on the device, outputs on the device).
cudaError_t mlp_forward(symhss_mlp_s* n, const float* x, int B, float* out, cudaStream_t s) {
  for (int b0 = 0; b0 < B; b0 += n->max_batch) {
    const int cnt = B - b0 < n->max_batch ? B - b0 : n->max_batch;
    cudaError_t e = forward_chunk(n, x + (size_t)b0 * kW, cnt, s);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(out + (size_t)b0 * kW, act_buf(n, 2), (size_t)cnt * kW * sizeof(float),
                        cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace symhss

extern "C" {

int symhss_mlp_create(const float* params, int max_batch, symhss_mlp_t* out) {
  if (!out) return SYMHSS_ERR_INVALID;
  *out = nullptr;
  if (max_batch < 1 || max_batch > (1 << 20)) return SYMHSS_ERR_INVALID;
  symhss_mlp_s* n = new (std::nothrow) symhss_mlp_s();
  if (!n) return SYMHSS_ERR_NOMEM;
  n->max_batch = max_batch;
  const size_t pb = (size_t)kMlpParams * sizeof(float);
  cudaError_t e = cudaMalloc(&n->master, pb);
  if (e == cudaSuccess) e = cudaMalloc(&n->m, pb);
  if (e == cudaSuccess) e = cudaMalloc(&n->v, pb);
  if (e == cudaSuccess) e = cudaMalloc(&n->grad, pb);
  if (e == cudaSuccess) e = cudaMalloc(&n->w16, (size_t)kMlpParams * sizeof(__half));
  if (e == cudaSuccess) e = cudaMalloc(&n->act, (size_t)6 * max_batch * kW * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&n->loss, sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(n->m, 0, pb);
  if (e == cudaSuccess) e = cudaMemset(n->v, 0, pb);
  if (e == cudaSuccess) e = cudaMemset(n->grad, 0, pb);
  if (e == cudaSuccess) e = cudaMemset(n->master, 0, pb);
  if (e != cudaSuccess) {
    delete n;
    return to_status(e);
  }
  int rc = params ? symhss_mlp_set_params(n, params) : SYMHSS_OK;
  if (rc == SYMHSS_OK && !params) {
    to_half_kernel<<<(kMlpParams + 255) / 256, 256>>>(n->master, n->w16, kMlpParams);
    count_launches(1);
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) rc = to_status(e);
  }
  if (rc) {
    delete n;
    return rc;
  }
  *out = n;
  return SYMHSS_OK;
}

int symhss_mlp_set_params(symhss_mlp_t n, const float* params) {
  if (!n || !params) return SYMHSS_ERR_INVALID;
  for (int k = 0; k < kMlpParams; ++k)
    if (!std::isfinite(params[k])) return SYMHSS_ERR_INVALID;
  cudaError_t e = cudaMemcpy(n->master, params, (size_t)kMlpParams * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return to_status(e);
  to_half_kernel<<<(kMlpParams + 255) / 256, 256>>>(n->master, n->w16, kMlpParams);
  count_launches(1);
  e = cudaMemset(n->m, 0, (size_t)kMlpParams * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(n->v, 0, (size_t)kMlpParams * sizeof(float));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  n->step = 0;
  return e == cudaSuccess ? SYMHSS_OK : to_status(e);
}

int symhss_mlp_get_params(symhss_mlp_t n, float* params, void* fp16_params) {
  if (!n || (!params && !fp16_params)) return SYMHSS_ERR_INVALID;
  cudaError_t e = cudaSuccess;
  if (params) e = cudaMemcpy(params, n->master, (size_t)kMlpParams * sizeof(float), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && fp16_params)
    e = cudaMemcpy(fp16_params, n->w16, (size_t)kMlpParams * sizeof(__half), cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? SYMHSS_OK : to_status(e);
}

int symhss_mlp_forward(symhss_mlp_t n, const float* x, int batch, float* out, void* stream) {
  if (!n || batch < 0 || (batch > 0 && (!x || !out))) return SYMHSS_ERR_INVALID;
  if (batch == 0) return SYMHSS_OK;
  cudaError_t e = mlp_forward(n, x, batch, out, (cudaStream_t)stream);
  return e == cudaSuccess ? SYMHSS_OK : to_status(e);
}

int symhss_mlp_loss_grad(symhss_mlp_t n, const float* x, const float* y_rank, const float* y_skel, const float* mask,
                         int batch, double* loss, float* grad, void* stream) {
  if (!n || !x || !y_rank || !y_skel || !mask || batch < 1 || batch > n->max_batch) return SYMHSS_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = loss_grad_chunk(n, x, y_rank, y_skel, mask, batch, s);
  if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, n->loss, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && grad)
    e = cudaMemcpyAsync(grad, n->grad, (size_t)kMlpParams * sizeof(float), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && (loss || grad)) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? SYMHSS_OK : to_status(e);
}

int symhss_mlp_train_step(symhss_mlp_t n, const float* x, const float* y_rank, const float* y_skel, const float* mask,
                          int batch, float lr, double* loss, void* stream) {
  if (!n || !x || !y_rank || !y_skel || !mask || batch < 1 || batch > n->max_batch) return SYMHSS_ERR_INVALID;
  if (!(lr > 0.0f) || !std::isfinite(lr)) return SYMHSS_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = loss_grad_chunk(n, x, y_rank, y_skel, mask, batch, s);
  if (e != cudaSuccess) return to_status(e);
  n->step += 1;
  const float c1 = (float)(1.0 - std::pow(0.9, (double)n->step));
  const float c2 = (float)(1.0 - std::pow(0.999, (double)n->step));
  adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, s>>>(n->master, n->m, n->v, n->grad, n->w16, kMlpParams, lr, c1, c2);
  count_launches(1);
  e = cudaGetLastError();
  if (e == cudaSuccess && loss) {
    e = cudaMemcpyAsync(loss, n->loss, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  return e == cudaSuccess ? SYMHSS_OK : to_status(e);
}

int symhss_mlp_destroy(symhss_mlp_t n) {
  delete n;
  return SYMHSS_OK;
}

}  // extern "C"
