// learned.cu -- the learned proposal's encoder: forward, backward, InfoNCE
// loss and AdamW, as hand-written kernels. Not part of the paper's method:
// the encoder maps a level-J data event (or a masked TI window) to a unit
// 64-vector so that a nearest-neighbour pass can propose candidates that the
// exact CCF of Eq. CCW then re-ranks.
//
// Network (input C x tj x tj, C = facies count channels scaled to [0, 1]):
//   conv 3x3 C->32 pad 1, ReLU; conv 3x3 32->32 stride 2 pad 1, ReLU;
//   conv 3x3 32->32 stride 2 pad 1, ReLU; linear (32 h3 h3)->64;
//   L2 normalisation.
// Parameters are FP32 masters; with `bf16` set, the forward and backward
// passes use the weights and store the activations rounded to BF16 (FP32
// arithmetic), as in BF16 mixed-precision training.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "ccw_internal.cuh"
#include "net_shape.cuh"

namespace ccw {

__device__ __forceinline__ float round_bf16(float v, int bf16) {
  return bf16 ? __bfloat162float(__float2bfloat16_rn(v)) : v;
}

// y[n][co][oy][ox] = relu(b[co] + sum_{ci,ky,kx} w[co][ci][ky][kx] x[n][ci][iy][ix])
__global__ void k_conv_fwd(const float* __restrict__ x, const float* __restrict__ w,
                           const float* __restrict__ b, float* __restrict__ y, int N, int Ci,
                           int H, int W, int Co, int Ho, int Wo, int stride, int relu, int bf16) {
  const int64_t total = (int64_t)N * Co * Ho * Wo;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int ox = (int)(i % Wo);
    const int oy = (int)((i / Wo) % Ho);
    const int co = (int)((i / ((int64_t)Wo * Ho)) % Co);
    const int n = (int)(i / ((int64_t)Wo * Ho * Co));
    float acc = b[co];
    for (int ci = 0; ci < Ci; ++ci)
      for (int ky = 0; ky < 3; ++ky) {
        const int iy = oy * stride + ky - 1;
        if (iy < 0 || iy >= H) continue;
        for (int kx = 0; kx < 3; ++kx) {
          const int ix = ox * stride + kx - 1;
          if (ix < 0 || ix >= W) continue;
          acc += round_bf16(w[((co * Ci + ci) * 3 + ky) * 3 + kx], bf16) *
                 x[(((int64_t)n * Ci + ci) * H + iy) * W + ix];
        }
      }
    if (relu && acc < 0.f) acc = 0.f;
    y[i] = round_bf16(acc, bf16);
  }
}

// dx[n][ci][iy][ix] = sum over the outputs that read (iy, ix) of
// w * dy * [y > 0]  (ReLU derivative taken from the stored output)
__global__ void k_conv_bwd_data(const float* __restrict__ dy, const float* __restrict__ y,
                                const float* __restrict__ w, float* __restrict__ dx, int N, int Ci,
                                int H, int W, int Co, int Ho, int Wo, int stride, int relu,
                                int bf16) {
  const int64_t total = (int64_t)N * Ci * H * W;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int ix = (int)(i % W);
    const int iy = (int)((i / W) % H);
    const int ci = (int)((i / ((int64_t)W * H)) % Ci);
    const int n = (int)(i / ((int64_t)W * H * Ci));
    float acc = 0.f;
    for (int ky = 0; ky < 3; ++ky) {
      const int t = iy + 1 - ky;   // = oy * stride
      if (t < 0 || t % stride) continue;
      const int oy = t / stride;
      if (oy >= Ho) continue;
      for (int kx = 0; kx < 3; ++kx) {
        const int u = ix + 1 - kx;
        if (u < 0 || u % stride) continue;
        const int ox = u / stride;
        if (ox >= Wo) continue;
        for (int co = 0; co < Co; ++co) {
          const int64_t o = (((int64_t)n * Co + co) * Ho + oy) * Wo + ox;
          if (relu && y[o] <= 0.f) continue;
          acc += round_bf16(w[((co * Ci + ci) * 3 + ky) * 3 + kx], bf16) * dy[o];
        }
      }
    }
    dx[i] = acc;
  }
}

// dw[co][ci][ky][kx] += sum_{n,oy,ox} dy' x ; db[co] += sum dy'  (dy' = dy [y > 0])
__global__ void k_conv_bwd_w(const float* __restrict__ dy, const float* __restrict__ y,
                             const float* __restrict__ x, float* __restrict__ dw,
                             float* __restrict__ db, int N, int Ci, int H, int W, int Co, int Ho,
                             int Wo, int stride, int relu) {
  const int nw = Co * Ci * 9;
  const int total = nw + Co;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    double acc = 0.0;
    if (i < nw) {
      const int kx = i % 3, ky = (i / 3) % 3, ci = (i / 9) % Ci, co = i / (9 * Ci);
      for (int n = 0; n < N; ++n)
        for (int oy = 0; oy < Ho; ++oy) {
          const int iy = oy * stride + ky - 1;
          if (iy < 0 || iy >= H) continue;
          for (int ox = 0; ox < Wo; ++ox) {
            const int ix = ox * stride + kx - 1;
            if (ix < 0 || ix >= W) continue;
            const int64_t o = (((int64_t)n * Co + co) * Ho + oy) * Wo + ox;
            if (relu && y[o] <= 0.f) continue;
            acc += (double)dy[o] * x[(((int64_t)n * Ci + ci) * H + iy) * W + ix];
          }
        }
      dw[i] += (float)acc;
    } else {
      const int co = i - nw;
      for (int n = 0; n < N; ++n)
        for (int p = 0; p < Ho * Wo; ++p) {
          const int64_t o = ((int64_t)n * Co + co) * Ho * Wo + p;
          if (relu && y[o] <= 0.f) continue;
          acc += dy[o];
        }
      db[co] += (float)acc;
    }
  }
}

// y[n][j] = b[j] + sum_k w[j][k] x[n][k]
__global__ void k_linear_fwd(const float* __restrict__ x, const float* __restrict__ w,
                             const float* __restrict__ b, float* __restrict__ y, int N, int In,
                             int Out, int bf16) {
  const int total = N * Out;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int j = i % Out, n = i / Out;
    float acc = b[j];
    for (int k = 0; k < In; ++k) acc += round_bf16(w[j * In + k], bf16) * x[(int64_t)n * In + k];
    y[i] = acc;
  }
}

__global__ void k_linear_bwd_data(const float* __restrict__ dy, const float* __restrict__ w,
                                  float* __restrict__ dx, int N, int In, int Out, int bf16) {
  const int total = N * In;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int k = i % In, n = i / In;
    float acc = 0.f;
    for (int j = 0; j < Out; ++j) acc += round_bf16(w[j * In + k], bf16) * dy[(int64_t)n * Out + j];
    dx[i] = acc;
  }
}

__global__ void k_linear_bwd_w(const float* __restrict__ dy, const float* __restrict__ x,
                               float* __restrict__ dw, float* __restrict__ db, int N, int In,
                               int Out) {
  const int total = Out * In + Out;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    double acc = 0.0;
    if (i < Out * In) {
      const int k = i % In, j = i / In;
      for (int n = 0; n < N; ++n) acc += (double)dy[(int64_t)n * Out + j] * x[(int64_t)n * In + k];
      dw[i] += (float)acc;
    } else {
      const int j = i - Out * In;
      for (int n = 0; n < N; ++n) acc += dy[(int64_t)n * Out + j];
      db[j] += (float)acc;
    }
  }
}

// e = z / |z| per row of D (one warp per row)
__global__ void k_l2norm_fwd(const float* __restrict__ z, float* __restrict__ e,
                             float* __restrict__ norm, int N, int D) {
  const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (row >= N) return;
  float s = 0.f;
  for (int k = lane; k < D; k += 32) s += z[(int64_t)row * D + k] * z[(int64_t)row * D + k];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  const float nr = sqrtf(fmaxf(s, 1e-24f));
  if (lane == 0) norm[row] = nr;
  for (int k = lane; k < D; k += 32) e[(int64_t)row * D + k] = z[(int64_t)row * D + k] / nr;
}

// dz = (de - e (e . de)) / |z|
__global__ void k_l2norm_bwd(const float* __restrict__ e, const float* __restrict__ norm,
                             const float* __restrict__ de, float* __restrict__ dz, int N, int D) {
  const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (row >= N) return;
  float s = 0.f;
  for (int k = lane; k < D; k += 32) s += e[(int64_t)row * D + k] * de[(int64_t)row * D + k];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  for (int k = lane; k < D; k += 32)
    dz[(int64_t)row * D + k] =
        (de[(int64_t)row * D + k] - e[(int64_t)row * D + k] * s) / norm[row];
}

// InfoNCE: logits[i][j] = a_i . c_j / tau over B anchors and M candidates,
// the positive of anchor i is candidate i. One CTA per anchor computes its
// loss term and the softmax; dA and the per-anchor contribution to dC follow.
__global__ void k_infonce(const float* __restrict__ A, const float* __restrict__ Cm, int B,
                          int M, int D, float tau, float* __restrict__ prob,
                          float* __restrict__ loss_terms) {
  extern __shared__ float sh[];   // M logits
  const int i = blockIdx.x;
  for (int j = threadIdx.x; j < M; j += blockDim.x) {
    float s = 0.f;
    for (int k = 0; k < D; ++k) s += A[(int64_t)i * D + k] * Cm[(int64_t)j * D + k];
    sh[j] = s / tau;
  }
  __syncthreads();
  __shared__ float red[33];
  float mx = -INFINITY;
  for (int j = threadIdx.x; j < M; j += blockDim.x) mx = fmaxf(mx, sh[j]);
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = -INFINITY;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) m = fmaxf(m, red[w]);
    red[32] = m;
  }
  __syncthreads();
  mx = red[32];
  __syncthreads();
  float se = 0.f;
  for (int j = threadIdx.x; j < M; j += blockDim.x) se += expf(sh[j] - mx);
  for (int o = 16; o > 0; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = se;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) s += red[w];
    red[32] = s;
  }
  __syncthreads();
  const float sum = red[32];
  for (int j = threadIdx.x; j < M; j += blockDim.x)
    prob[(int64_t)i * M + j] = expf(sh[j] - mx) / sum;
  if (threadIdx.x == 0) loss_terms[i] = -(sh[i] - mx - logf(sum));
}

// dL/dlogits = (prob - onehot) / B; dA = dlogits C / tau; dC = dlogits^T A / tau
__global__ void k_infonce_bwd_a(const float* __restrict__ prob, const float* __restrict__ Cm,
                                float* __restrict__ dA, int B, int M, int D, float tau) {
  const int total = B * D;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int k = t % D, i = t / D;
    float acc = 0.f;
    for (int j = 0; j < M; ++j) {
      const float g = (prob[(int64_t)i * M + j] - (i == j ? 1.f : 0.f)) / B;
      acc += g * Cm[(int64_t)j * D + k];
    }
    dA[t] = acc / tau;
  }
}

__global__ void k_infonce_bwd_c(const float* __restrict__ prob, const float* __restrict__ A,
                                float* __restrict__ dC, int B, int M, int D, float tau) {
  const int total = M * D;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int k = t % D, j = t / D;
    float acc = 0.f;
    for (int i = 0; i < B; ++i) {
      const float g = (prob[(int64_t)i * M + j] - (i == j ? 1.f : 0.f)) / B;
      acc += g * A[(int64_t)i * D + k];
    }
    dC[t] = acc / tau;
  }
}

__global__ void k_mean(const float* __restrict__ v, int n, float* __restrict__ out) {
  __shared__ float red[32];
  float s = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += v[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += red[w];
    *out = t / n;
  }
}

// AdamW (decoupled weight decay) on the FP32 masters.
__global__ void k_adamw(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                        float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps,
                        float wd, float bc1, float bc2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / bc1, vh = vi / bc2;
    p[i] -= lr * (mh / (sqrtf(vh) + eps) + wd * p[i]);
  }
}

}  // namespace ccw

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace ccw {

int64_t infer_act_floats(int C, int tj);
// Inference pass (defined below): see net_infer.
cudaError_t net_infer(const float* P, int C, int tj, const float* x, int N, float* act,
                      float* emb, cudaStream_t st, int* status, int path, const void* wimg);

static int grid_for(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 152 * 16); }

}  // namespace ccw

using namespace ccw;

struct ccw_net {
  NetShape s;
  float* p = nullptr;   // FP32 master parameters
  float* g = nullptr;   // gradients
  float* m = nullptr;   // AdamW moments
  float* v = nullptr;
  int64_t step = 0;
  // activations of the last forward pass (capacity in samples)
  int cap = 0;
  float *a1 = nullptr, *a2 = nullptr, *a3 = nullptr, *z = nullptr, *e = nullptr, *nrm = nullptr;
  float *d1 = nullptr, *d2 = nullptr, *d3 = nullptr, *dz = nullptr, *de = nullptr;
  float *prob = nullptr, *lterm = nullptr;
  int prob_cap = 0;
};

namespace {
thread_local char g_net_err[256] = "";
int net_fail(int code, const char* msg) {
  snprintf(g_net_err, sizeof(g_net_err), "%s", msg);
  return code;
}

void free_acts(ccw_net* n) {
  for (float** q : {&n->a1, &n->a2, &n->a3, &n->z, &n->e, &n->nrm, &n->d1, &n->d2, &n->d3, &n->dz,
                    &n->de}) {
    cudaFree(*q);
    *q = nullptr;
  }
  n->cap = 0;
}

int ensure_acts(ccw_net* n, int N) {
  if (N <= n->cap) return CCW_OK;
  free_acts(n);
  const NetShape& s = n->s;
  const int64_t s1 = 32LL * s.tj * s.tj, s2 = 32LL * s.h2 * s.h2, s3 = 32LL * s.h3 * s.h3;
  cudaError_t e = cudaSuccess;
  auto al = [&](float** q, int64_t cnt) {
    if (e == cudaSuccess) e = cudaMalloc(q, sizeof(float) * std::max<int64_t>(cnt, 1));
  };
  al(&n->a1, N * s1);
  al(&n->a2, N * s2);
  al(&n->a3, N * s3);
  al(&n->z, N * 64LL);
  al(&n->e, N * 64LL);
  al(&n->nrm, N);
  al(&n->d1, N * s1);
  al(&n->d2, N * s2);
  al(&n->d3, N * s3);
  al(&n->dz, N * 64LL);
  al(&n->de, N * 64LL);
  if (e != cudaSuccess) {
    free_acts(n);
    return net_fail(CCW_ENOMEM, "encoder activations");
  }
  n->cap = N;
  return CCW_OK;
}

// forward pass of N samples into n->e (unit embeddings)
void net_forward(ccw_net* n, const float* x, int N, int bf16, cudaStream_t st) {
  const NetShape& s = n->s;
  const float* P = n->p;
  k_conv_fwd<<<grid_for((int64_t)N * 32 * s.tj * s.tj), 256, 0, st>>>(
      x, P + s.o_w1, P + s.o_b1, n->a1, N, s.C, s.tj, s.tj, 32, s.tj, s.tj, 1, 1, bf16);
  k_conv_fwd<<<grid_for((int64_t)N * 32 * s.h2 * s.h2), 256, 0, st>>>(
      n->a1, P + s.o_w2, P + s.o_b2, n->a2, N, 32, s.tj, s.tj, 32, s.h2, s.h2, 2, 1, bf16);
  k_conv_fwd<<<grid_for((int64_t)N * 32 * s.h3 * s.h3), 256, 0, st>>>(
      n->a2, P + s.o_w3, P + s.o_b3, n->a3, N, 32, s.h2, s.h2, 32, s.h3, s.h3, 2, 1, bf16);
  k_linear_fwd<<<grid_for((int64_t)N * 64), 256, 0, st>>>(n->a3, P + s.o_wf, P + s.o_bf, n->z, N,
                                                          s.flat, 64, bf16);
  k_l2norm_fwd<<<(N + 7) / 8, 256, 0, st>>>(n->z, n->e, n->nrm, N, 64);
}

// backward of N samples from n->de (gradient wrt the unit embeddings),
// accumulating into n->g
void net_backward(ccw_net* n, const float* x, int N, int bf16, cudaStream_t st) {
  const NetShape& s = n->s;
  const float* P = n->p;
  float* G = n->g;
  k_l2norm_bwd<<<(N + 7) / 8, 256, 0, st>>>(n->e, n->nrm, n->de, n->dz, N, 64);
  k_linear_bwd_w<<<grid_for(64LL * s.flat + 64), 256, 0, st>>>(n->dz, n->a3, G + s.o_wf,
                                                              G + s.o_bf, N, s.flat, 64);
  k_linear_bwd_data<<<grid_for((int64_t)N * s.flat), 256, 0, st>>>(n->dz, P + s.o_wf, n->d3, N,
                                                                  s.flat, 64, bf16);
  k_conv_bwd_w<<<grid_for(32LL * 32 * 9 + 32), 256, 0, st>>>(
      n->d3, n->a3, n->a2, G + s.o_w3, G + s.o_b3, N, 32, s.h2, s.h2, 32, s.h3, s.h3, 2, 1);
  k_conv_bwd_data<<<grid_for((int64_t)N * 32 * s.h2 * s.h2), 256, 0, st>>>(
      n->d3, n->a3, P + s.o_w3, n->d2, N, 32, s.h2, s.h2, 32, s.h3, s.h3, 2, 1, bf16);
  k_conv_bwd_w<<<grid_for(32LL * 32 * 9 + 32), 256, 0, st>>>(
      n->d2, n->a2, n->a1, G + s.o_w2, G + s.o_b2, N, 32, s.tj, s.tj, 32, s.h2, s.h2, 2, 1);
  k_conv_bwd_data<<<grid_for((int64_t)N * 32 * s.tj * s.tj), 256, 0, st>>>(
      n->d2, n->a2, P + s.o_w2, n->d1, N, 32, s.tj, s.tj, 32, s.h2, s.h2, 2, 1, bf16);
  k_conv_bwd_w<<<grid_for(32LL * s.C * 9 + 32), 256, 0, st>>>(
      n->d1, n->a1, x, G + s.o_w1, G + s.o_b1, N, s.C, s.tj, s.tj, 32, s.tj, s.tj, 1, 1);
}

}  // namespace

extern "C" {

const char* ccw_net_last_error(void) { return g_net_err; }

int ccw_net_create(int32_t in_ch, int32_t tj, uint64_t seed, ccw_net** out) {
  if (!out) return net_fail(CCW_EINVAL, "out is NULL");
  *out = nullptr;
  if (in_ch < 1 || in_ch > 16 || tj < 3 || tj > 64)
    return net_fail(CCW_EINVAL, "in_ch must be in [1, 16] and tj in [3, 64]");
  ccw_net* n = new ccw_net();
  n->s = net_shape(in_ch, tj);
  const int64_t np = n->s.n;
  cudaError_t e = cudaSuccess;
  for (float** q : {&n->p, &n->g, &n->m, &n->v})
    if (e == cudaSuccess) e = cudaMalloc(q, sizeof(float) * np);
  if (e != cudaSuccess) {
    for (float* q : {n->p, n->g, n->m, n->v}) cudaFree(q);
    delete n;
    return net_fail(CCW_ENOMEM, "encoder parameters");
  }
  // He-normal weights from a seeded generator (splitmix64 + Box-Muller),
  // zero biases
  std::vector<float> h(np, 0.f);
  uint64_t st = seed ^ 0x9E3779B97F4A7C15ull;
  auto next = [&]() {
    st += 0x9E3779B97F4A7C15ull;
    uint64_t z = st;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
  };
  auto fill = [&](int64_t off, int64_t cnt, double fan_in) {
    const double sd = std::sqrt(2.0 / fan_in);
    for (int64_t i = 0; i < cnt; ++i) {
      const double u1 = std::max(next(), 1e-300), u2 = next();
      h[off + i] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
    }
  };
  const NetShape& s = n->s;
  fill(s.o_w1, 32LL * in_ch * 9, in_ch * 9.0);
  fill(s.o_w2, 32LL * 32 * 9, 32 * 9.0);
  fill(s.o_w3, 32LL * 32 * 9, 32 * 9.0);
  fill(s.o_wf, 64LL * s.flat, s.flat);
  cudaMemcpy(n->p, h.data(), sizeof(float) * np, cudaMemcpyHostToDevice);
  cudaMemset(n->g, 0, sizeof(float) * np);
  cudaMemset(n->m, 0, sizeof(float) * np);
  cudaMemset(n->v, 0, sizeof(float) * np);
  *out = n;
  return CCW_OK;
}

void ccw_net_free(ccw_net* n) {
  if (!n) return;
  cudaDeviceSynchronize();
  free_acts(n);
  for (float* q : {n->p, n->g, n->m, n->v, n->prob, n->lterm}) cudaFree(q);
  delete n;
}

int64_t ccw_net_param_count(const ccw_net* n) { return n ? n->s.n : -1; }

int ccw_net_get(const ccw_net* n, int32_t what, float* host) {
  if (!n || !host) return net_fail(CCW_EINVAL, "NULL argument");
  const float* src = what == 0 ? n->p : what == 1 ? n->g : nullptr;
  if (!src) return net_fail(CCW_EINVAL, "what must be 0 (parameters) or 1 (gradients)");
  if (cudaMemcpy(host, src, sizeof(float) * n->s.n, cudaMemcpyDeviceToHost) != cudaSuccess)
    return net_fail(CCW_ECUDA, "copy");
  return CCW_OK;
}

int ccw_net_set(ccw_net* n, const float* host) {
  if (!n || !host) return net_fail(CCW_EINVAL, "NULL argument");
  if (cudaMemcpy(n->p, host, sizeof(float) * n->s.n, cudaMemcpyHostToDevice) != cudaSuccess)
    return net_fail(CCW_ECUDA, "copy");
  return CCW_OK;
}

int ccw_net_embed(ccw_net* n, const float* x_dev, int32_t N, int32_t bf16, float* emb_dev,
                  void* stream) {
  if (!n || (!x_dev && N > 0) || (!emb_dev && N > 0) || N < 0)
    return net_fail(CCW_EINVAL, "bad argument");
  if (N == 0) return CCW_OK;
  cudaStream_t st = (cudaStream_t)stream;
  if (bf16 == 2 || bf16 == 3) {
    // the inference pass of the proposal (2: tensor cores where the shape
    // fits; 3: the FP32-lane kernels), with scratch for the per-layer path
    float* act = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&act,
                                    sizeof(float) * (size_t)infer_act_floats(n->s.C, n->s.tj) * N,
                                    st);
    if (e != cudaSuccess) return net_fail(CCW_ENOMEM, "inference scratch");
    e = net_infer(n->p, n->s.C, n->s.tj, x_dev, N, act, emb_dev, st, nullptr, bf16 == 3 ? 1 : 0,
                  nullptr);
    cudaFreeAsync(act, st);
    if (e != cudaSuccess) return net_fail(CCW_ECUDA, "inference kernel");
    return CCW_OK;
  }
  for (int i0 = 0; i0 < N; i0 += 4096) {
    const int c = std::min(4096, N - i0);
    if (int rc = ensure_acts(n, c)) return rc;
    net_forward(n, x_dev + (int64_t)i0 * n->s.C * n->s.tj * n->s.tj, c, bf16, st);
    if (cudaMemcpyAsync(emb_dev + (int64_t)i0 * 64, n->e, sizeof(float) * c * 64,
                        cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return net_fail(CCW_ECUDA, "embedding copy");
  }
  if (cudaGetLastError() != cudaSuccess) return net_fail(CCW_ECUDA, "encoder kernels");
  return CCW_OK;
}

int ccw_net_train_step(ccw_net* n, const float* anchors_dev, int32_t B, const float* cands_dev,
                       int32_t M, float tau, float lr, float wd, int32_t bf16, int32_t apply,
                       float* loss_dev, void* stream) {
  if (!n || !anchors_dev || !cands_dev || B < 1 || M < B || tau <= 0.f)
    return net_fail(CCW_EINVAL, "bad argument (need B >= 1, M >= B, tau > 0)");
  cudaStream_t st = (cudaStream_t)stream;
  const NetShape& s = n->s;
  const int64_t in_sz = (int64_t)s.C * s.tj * s.tj;
  const int N = B + M;
  if (int rc = ensure_acts(n, N)) return rc;
  if (B * M > n->prob_cap) {
    cudaFree(n->prob);
    cudaFree(n->lterm);
    n->prob = nullptr;
    n->lterm = nullptr;
    if (cudaMalloc(&n->prob, sizeof(float) * (int64_t)B * M) != cudaSuccess ||
        cudaMalloc(&n->lterm, sizeof(float) * B) != cudaSuccess)
      return net_fail(CCW_ENOMEM, "loss buffers");
    n->prob_cap = B * M;
  }
  // one forward over [anchors; candidates] (shared weights)
  float* x = nullptr;
  if (cudaMallocAsync(&x, sizeof(float) * N * in_sz, st) != cudaSuccess)
    return net_fail(CCW_ENOMEM, "input staging");
  cudaMemcpyAsync(x, anchors_dev, sizeof(float) * B * in_sz, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(x + (int64_t)B * in_sz, cands_dev, sizeof(float) * M * in_sz,
                  cudaMemcpyDeviceToDevice, st);
  net_forward(n, x, N, bf16, st);
  const float* EA = n->e;
  const float* EC = n->e + (int64_t)B * 64;
  k_infonce<<<B, 256, sizeof(float) * M, st>>>(EA, EC, B, M, 64, tau, n->prob, n->lterm);
  if (loss_dev) k_mean<<<1, 256, 0, st>>>(n->lterm, B, loss_dev);
  k_infonce_bwd_a<<<grid_for((int64_t)B * 64), 256, 0, st>>>(n->prob, EC, n->de, B, M, 64, tau);
  k_infonce_bwd_c<<<grid_for((int64_t)M * 64), 256, 0, st>>>(n->prob, EA, n->de + (int64_t)B * 64,
                                                            B, M, 64, tau);
  cudaMemsetAsync(n->g, 0, sizeof(float) * s.n, st);
  net_backward(n, x, N, bf16, st);
  cudaFreeAsync(x, st);
  if (apply) {
    ++n->step;
    const float b1 = 0.9f, b2 = 0.999f;
    const float bc1 = 1.f - (float)std::pow(b1, (double)n->step);
    const float bc2 = 1.f - (float)std::pow(b2, (double)n->step);
    k_adamw<<<grid_for(s.n), 256, 0, st>>>(n->p, n->g, n->m, n->v, s.n, lr, b1, b2, 1e-8f, wd,
                                           bc1, bc2);
  }
  if (cudaGetLastError() != cudaSuccess) return net_fail(CCW_ECUDA, "training kernels");
  return CCW_OK;
}

}  // extern "C"

namespace ccw {
// Shape and parameters of a network, for the proposal tables of a TI.
void net_view(const ccw_net* n, int* C, int* tj, const float** params, int64_t* count) {
  *C = n->s.C;
  *tj = n->s.tj;
  *params = n->p;
  *count = n->s.n;
}
}  // namespace ccw

namespace ccw {
// Inference forward pass of the encoder on N samples x [N][C][tj][tj]
// (BF16 weights and activations, the passes of training with bf16 = 1):
// act holds N * infer_act_floats(C, tj) floats of scratch, emb receives the
// unit embeddings [N][64]. Batched over all samples of a step: every layer
// is one grid-wide launch.
int64_t infer_act_floats(int C, int tj) {
  const NetShape s = net_shape(C, tj);
  return 32LL * tj * tj + 32LL * s.h2 * s.h2 + s.flat + 64 + 1;
}

// BF16 value of a 16-bit pattern (the weights are BF16-rounded when staged)
__device__ __forceinline__ float bf16_at(const uint16_t* w, int i) {
  return __uint_as_float((uint32_t)w[i] << 16);
}

// One 3 x 3 convolution layer (pad 1) of one sample in shared memory:
// y[co][oy][ox] = round_bf16(relu(b[co] + sum_{ci,ky,kx} round_bf16(w) x)),
// each output summed in the order of k_conv_fwd (bias first, then ci, ky, kx)
// so that the result is the same bit for bit. The weights are staged
// channel-minor, wt[((ci * 3 + ky) * 3 + kx) * 32 + co] (BF16), so that one
// 8-byte load serves the 4 output channels a thread computes.
__device__ __forceinline__ void conv_layer_smem(const float* __restrict__ x, int Ci, int H, int W,
                                                const uint16_t* __restrict__ wt,
                                                const float* __restrict__ b, float* y, int Ho,
                                                int Wo, int stride) {
  const int npix = Ho * Wo;
  for (int i = threadIdx.x; i < npix * 8; i += blockDim.x) {
    const int pix = i % npix, co0 = (i / npix) * 4;
    const int oy = pix / Wo, ox = pix % Wo;
    float acc[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[c] = __ldg(b + co0 + c);
    for (int ci = 0; ci < Ci; ++ci)
      for (int ky = 0; ky < 3; ++ky) {
        const int iy = oy * stride + ky - 1;
        if (iy < 0 || iy >= H) continue;
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) {
          const int ix = ox * stride + kx - 1;
          if (ix < 0 || ix >= W) continue;
          const float xv = x[(ci * H + iy) * W + ix];
          const uint2 w4 = *reinterpret_cast<const uint2*>(wt + ((ci * 3 + ky) * 3 + kx) * 32 + co0);
          acc[0] += __uint_as_float(w4.x << 16) * xv;
          acc[1] += __uint_as_float(w4.x & 0xFFFF0000u) * xv;
          acc[2] += __uint_as_float(w4.y << 16) * xv;
          acc[3] += __uint_as_float(w4.y & 0xFFFF0000u) * xv;
        }
      }
#pragma unroll
    for (int c = 0; c < 4; ++c)
      y[((co0 + c) * Ho + oy) * Wo + ox] = round_bf16(acc[c] < 0.f ? 0.f : acc[c], 1);
  }
}

// Stages conv weights w[co][ci][3][3] (FP32 masters) as BF16 in the
// channel-minor layout of conv_layer_smem.
// Reads w[0 .. n) in its own (contiguous) order, 8 loads in flight per
// thread, and stores element i at dst[perm(i)] as BF16.
template <typename Perm>
__device__ __forceinline__ void stage_bf16(const float* __restrict__ w, int n, uint16_t* dst,
                                           Perm perm) {
  for (int i0 = threadIdx.x; i0 < n; i0 += 8 * blockDim.x) {
    float v[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int i = i0 + b * blockDim.x;
      v[b] = i < n ? __ldg(w + i) : 0.f;
    }
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int i = i0 + b * blockDim.x;
      if (i < n) dst[perm(i)] = __bfloat16_as_ushort(__float2bfloat16_rn(v[b]));
    }
  }
}

// Stages conv weights w[co][ci][3][3] (FP32 masters) as BF16 in the
// channel-minor layout of conv_layer_smem.
__device__ __forceinline__ void stage_conv_weights(const float* __restrict__ w, int Ci,
                                                   uint16_t* wt) {
  const int per = Ci * 9;   // r = (ci * 3 + ky) * 3 + kx
  stage_bf16(w, 32 * per, wt, [per](int i) { return (i % per) * 32 + i / per; });
}

// The whole inference forward pass of the encoder, samples taken in turn by
// each CTA, activations and BF16 weights in shared memory (the weights staged
// once per CTA); the same arithmetic as the layer-by-layer kernels
// (k_conv_fwd x 3, k_linear_fwd, k_l2norm_fwd with bf16 = 1).
__global__ void __launch_bounds__(256) k_encode_fused(const float* __restrict__ P, NetShape s,
                                                      const float* __restrict__ x, int N,
                                                      float* __restrict__ emb) {
  extern __shared__ float sh[];
  const int tj = s.tj, C = s.C;
  float* xs = sh;                                   // [C][tj][tj]
  float* a1 = xs + C * tj * tj;                     // [32][tj][tj]
  float* a2 = a1 + 32 * tj * tj;                    // [32][h2][h2]
  float* a3 = a2 + 32 * s.h2 * s.h2;                // [flat]
  float* z = a3 + s.flat;                           // [64]
  // the BF16 weights start 16-byte aligned (8-byte loads of 4 channels)
  const int act_floats = (C * tj * tj + 32 * tj * tj + 32 * s.h2 * s.h2 + s.flat + 64 + 3) & ~3;
  uint16_t* w1 = reinterpret_cast<uint16_t*>(sh + act_floats);   // [C*9][32]
  uint16_t* w2 = w1 + 32 * C * 9;                   // [32*9][32]
  uint16_t* w3 = w2 + 32 * 32 * 9;                  // [32*9][32]
  uint16_t* wf = w3 + 32 * 32 * 9;                  // [flat][64]
  stage_conv_weights(P + s.o_w1, C, w1);
  stage_conv_weights(P + s.o_w2, 32, w2);
  stage_conv_weights(P + s.o_w3, 32, w3);
  {
    const int flat = s.flat;   // wf[k][j] from the master's [j][k]
    stage_bf16(P + s.o_wf, 64 * flat, wf, [flat](int i) { return (i % flat) * 64 + i / flat; });
  }
  for (int n = blockIdx.x; n < N; n += gridDim.x) {
    const float* xn = x + (int64_t)n * C * tj * tj;
    for (int i = threadIdx.x; i < C * tj * tj; i += blockDim.x) xs[i] = __ldg(xn + i);
    __syncthreads();
    conv_layer_smem(xs, C, tj, tj, w1, P + s.o_b1, a1, tj, tj, 1);
    __syncthreads();
    conv_layer_smem(a1, 32, tj, tj, w2, P + s.o_b2, a2, s.h2, s.h2, 2);
    __syncthreads();
    conv_layer_smem(a2, 32, s.h2, s.h2, w3, P + s.o_b3, a3, s.h3, s.h3, 2);
    __syncthreads();
    for (int j = threadIdx.x; j < 64; j += blockDim.x) {
      float acc = __ldg(P + s.o_bf + j);
      for (int k = 0; k < s.flat; ++k) acc += bf16_at(wf, k * 64 + j) * a3[k];
      z[j] = acc;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      float q = 0.f;
      for (int k = lane; k < 64; k += 32) q += z[k] * z[k];
      for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
      const float nr = sqrtf(fmaxf(q, 1e-24f));
      for (int k = lane; k < 64; k += 32) emb[(int64_t)n * 64 + k] = z[k] / nr;
    }
    __syncthreads();   // the next sample reuses the buffers
  }
}

int encode_fused_smem(const NetShape& s);
// Does the fused FP32-lane inference kernel take shape (C, tj)?
bool net_infer_fused_fits(int C, int tj) { return encode_fused_smem(net_shape(C, tj)) <= 110 * 1024; }

// Shared-memory bytes of k_encode_fused: activations, then BF16 weights.
int encode_fused_smem(const NetShape& s) {
  const int act = (int)sizeof(float) *
                  ((s.C * s.tj * s.tj + 32 * s.tj * s.tj + 32 * s.h2 * s.h2 + s.flat + 64 + 3) &
                   ~3);
  const int w = 2 * (32 * s.C * 9 + 2 * 32 * 32 * 9 + 64 * s.flat);
  return act + ((w + 15) & ~15);
}

cudaError_t net_infer_tc(const float* P, const void* wimg, int C, int tj, const float* x, int N,
                         float* emb, int* status, cudaStream_t st);

// path 0: the tensor-core kernel where the shape fits (encoder_tc.cu; wimg
// its weight image or NULL), else the fused FP32-lane kernel, else one launch
// per layer (needs `act`); path 1: never the tensor cores.
cudaError_t net_infer(const float* P, int C, int tj, const float* x, int N, float* act,
                      float* emb, cudaStream_t st, int* status, int path, const void* wimg) {
  if (N <= 0) return cudaSuccess;
  if (path == 0) {
    const cudaError_t e = net_infer_tc(P, wimg, C, tj, x, N, emb, status, st);
    if (e != cudaErrorNotSupported) return e;
  }
  {
    // one CTA per sample with the activations in shared memory, when they fit
    const NetShape s = net_shape(C, tj);
    const int smem = encode_fused_smem(s);
    if (smem <= 110 * 1024) {
      if (smem > 48 * 1024 &&
          cudaFuncSetAttribute(k_encode_fused, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               smem) != cudaSuccess)
        return cudaGetLastError();
      // two CTAs per SM take the samples in turn (weights staged once each)
      static int sms = 0;
      if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
      }
      const int grid = N < 2 * sms ? N : 2 * sms;
      k_encode_fused<<<grid, 256, smem, st>>>(P, s, x, N, emb);
      return cudaGetLastError();
    }
  }
  if (!act) return cudaErrorInvalidValue;
  const NetShape s = net_shape(C, tj);
  float* a1 = act;
  float* a2 = a1 + (int64_t)N * 32 * tj * tj;
  float* a3 = a2 + (int64_t)N * 32 * s.h2 * s.h2;
  float* z = a3 + (int64_t)N * s.flat;
  float* nrm = z + (int64_t)N * 64;
  k_conv_fwd<<<grid_for((int64_t)N * 32 * tj * tj), 256, 0, st>>>(
      x, P + s.o_w1, P + s.o_b1, a1, N, C, tj, tj, 32, tj, tj, 1, 1, 1);
  k_conv_fwd<<<grid_for((int64_t)N * 32 * s.h2 * s.h2), 256, 0, st>>>(
      a1, P + s.o_w2, P + s.o_b2, a2, N, 32, tj, tj, 32, s.h2, s.h2, 2, 1, 1);
  k_conv_fwd<<<grid_for((int64_t)N * 32 * s.h3 * s.h3), 256, 0, st>>>(
      a2, P + s.o_w3, P + s.o_b3, a3, N, 32, s.h2, s.h2, 32, s.h3, s.h3, 2, 1, 1);
  k_linear_fwd<<<grid_for((int64_t)N * 64), 256, 0, st>>>(a3, P + s.o_wf, P + s.o_bf, z, N,
                                                          s.flat, 64, 1);
  k_l2norm_fwd<<<(N + 7) / 8, 256, 0, st>>>(z, emb, nrm, N, 64);
  return cudaGetLastError();
}
}  // namespace ccw

namespace ccw {
// Round the weights (not the biases) of an encoder to BF16 values in place:
// the inference passes then read BF16 weights without converting.
__global__ void k_round_weights(float* p, NetShape s) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < s.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const bool bias = (i >= s.o_b1 && i < s.o_b1 + 32) || (i >= s.o_b2 && i < s.o_b2 + 32) ||
                      (i >= s.o_b3 && i < s.o_b3 + 32) || i >= s.o_bf;
    if (!bias) p[i] = __bfloat162float(__float2bfloat16_rn(p[i]));
  }
}

cudaError_t launch_round_weights(float* p, int C, int tj, cudaStream_t st) {
  k_round_weights<<<64, 256, 0, st>>>(p, net_shape(C, tj));
  return cudaGetLastError();
}
}  // namespace ccw
