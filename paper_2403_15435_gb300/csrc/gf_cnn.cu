// Learned refinement predictor: a 3-layer convolutional network on 16 x 16
// downsampled patch features, BF16 operands on the tensor cores (warp-level
// mma m16n8k16) with FP32 accumulation, its backward pass and an Adam step.
//
// Network (per patch): x0 = features on an 18 x 18 grid, the 16 x 16 patch
// pixels and a one-pixel ring from beyond its edges ([324 px][16 ch]);
// a_1 = relu(conv3x3_valid(x0; W_1) + b_1) on the 16 x 16 pixels, a_l =
// relu(conv3x3(a_{l-1}; W_l) + b_l) with zero padding for l = 2, 3, 16
// channels each; v = mean over pixels of a_3; logit = wh . v + bh.
// Layouts: activations [patch][256][16] BF16 (pixel-major, pixel = y*16 +
// x); conv weights [16 co][144 k] with k = tap*16 + ci and tap = (dy+1)*3 +
// (dx+1).  Every conv is an implicit GEMM with M = 256 pixels, N = 16,
// K = 144; the weight gradient is a GEMM with M = 16, N = 144 and K =
// pixels x patches.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace {

using bf16 = __nv_bfloat16;
constexpr int NPIX = 256, NCH = 16, KK = 144, PADW = 18, NPAD = PADW * PADW;

__device__ __forceinline__ unsigned saddr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(saddr(p)));
}

__device__ __forceinline__ void ldsm_x4_t(unsigned (&r)[4], const void* p) {
  asm volatile(
      "ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
      : "r"(saddr(p)));
}

// D = A (16x16 bf16, row) * B (16x8 bf16, col) + D (f32)
__device__ __forceinline__ void mma16816(float (&d)[4], const unsigned (&a)[4],
                                         unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, "
      "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Stage one patch's activations into an 18 x 18 x 16 tile: the input grid
// itself when it carries its ring (HALO), else 16 x 16 with a zero border.
template <bool HALO>
__device__ void stage_padded(const bf16* __restrict__ src, bf16* tile) {
  uint4* t4 = reinterpret_cast<uint4*>(tile);  // 2 x uint4 per pixel
  const uint4* s4 = reinterpret_cast<const uint4*>(src);
  if (HALO) {
    for (int k = threadIdx.x; k < PADW * PADW * 2; k += blockDim.x) t4[k] = s4[k];
    return;
  }
  const uint4 z = make_uint4(0u, 0u, 0u, 0u);
  for (int k = threadIdx.x; k < PADW * PADW * 2; k += blockDim.x) t4[k] = z;
  __syncthreads();
  for (int k = threadIdx.x; k < NPIX * 2; k += blockDim.x) {
    const int pix = k >> 1, half = k & 1;
    const int y = pix >> 4, x = pix & 15;
    t4[((y + 1) * PADW + (x + 1)) * 2 + half] = s4[k];
  }
}

__device__ __forceinline__ const bf16* tap_row(const bf16* tile, int pix,
                                               int tap) {
  const int y = pix >> 4, x = pix & 15;
  const int dy = tap / 3 - 1, dx = tap % 3 - 1;
  return tile + ((y + dy + 1) * PADW + (x + dx + 1)) * NCH;
}

// Convolution layer (also the input-gradient pass with flipped weights):
// out[p][co] = sum_{tap,ci} W[co][tap*16+ci] * in[p + tap][ci] (+ bias),
// then relu, or multiplied by (mask > 0).  One CTA (8 warps) per patch.
template <bool BIAS, bool RELU, bool MASK, bool HALO>
__global__ void __launch_bounds__(256) k_conv(const bf16* __restrict__ in,
                                              const bf16* __restrict__ W,
                                              const float* __restrict__ bias,
                                              const bf16* __restrict__ mask,
                                              bf16* __restrict__ out) {
  __shared__ __align__(16) bf16 tile[PADW * PADW * NCH];
  __shared__ __align__(16) bf16 sw[NCH * KK];
  const int p = blockIdx.x;
  stage_padded<HALO>(in + (size_t)p * (HALO ? NPAD : NPIX) * NCH, tile);
  for (int k = threadIdx.x; k < NCH * KK / 8; k += blockDim.x)
    reinterpret_cast<uint4*>(sw)[k] = reinterpret_cast<const uint4*>(W)[k];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float acc[2][2][4] = {};
  for (int tap = 0; tap < 9; ++tap) {
    unsigned b[4];
    ldsm_x4(b, sw + ((lane & 7) + 8 * (lane >> 4)) * KK + tap * 16 +
                   8 * ((lane >> 3) & 1));
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const int pix = warp * 32 + mt * 16 + (lane & 7) + 8 * ((lane >> 3) & 1);
      unsigned a[4];
      ldsm_x4(a, tap_row(tile, pix, tap) + 8 * (lane >> 4));
      mma16816(acc[mt][0], a, b[0], b[1]);
      mma16816(acc[mt][1], a, b[2], b[3]);
    }
  }
  bf16* o = out + (size_t)p * NPIX * NCH;
  const bf16* mk = MASK ? mask + (size_t)p * NPIX * NCH : nullptr;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int pix = warp * 32 + mt * 16 + (lane >> 2) + 8 * h;
        const int co = nt * 8 + (lane & 3) * 2;
        float v0 = acc[mt][nt][2 * h], v1 = acc[mt][nt][2 * h + 1];
        if (BIAS) { v0 += bias[co]; v1 += bias[co + 1]; }
        if (RELU) { v0 = fmaxf(v0, 0.f); v1 = fmaxf(v1, 0.f); }
        if (MASK) {
          if (!(__bfloat162float(mk[pix * NCH + co]) > 0.f)) v0 = 0.f;
          if (!(__bfloat162float(mk[pix * NCH + co + 1]) > 0.f)) v1 = 0.f;
        }
        __nv_bfloat162 r;
        r.x = __float2bfloat16_rn(v0);
        r.y = __float2bfloat16_rn(v1);
        *reinterpret_cast<__nv_bfloat162*>(o + pix * NCH + co) = r;
      }
}

// Weight gradient of a layer: dW[co][tap*16+ci] += sum_p dY[p][co] *
// in[p + tap][ci] over the patches of this CTA (a GEMM with M = 16, N = 144,
// K = pixels); one warp per tap.  db[co] += sum_p dY[p][co].
template <bool HALO>
__global__ void __launch_bounds__(288) k_conv_dw(const bf16* __restrict__ dY,
                                                 const bf16* __restrict__ in,
                                                 float* __restrict__ dW,
                                                 float* __restrict__ db,
                                                 int npatch, int group) {
  __shared__ __align__(16) bf16 tile[PADW * PADW * NCH];
  __shared__ __align__(16) bf16 sdy[NPIX * NCH];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tap = warp;
  float acc[2][4] = {};
  float dbs = 0.f;
  const int p0 = blockIdx.x * group;
  for (int pp = p0; pp < p0 + group && pp < npatch; ++pp) {
    __syncthreads();
    stage_padded<HALO>(in + (size_t)pp * (HALO ? NPAD : NPIX) * NCH, tile);
    for (int k = threadIdx.x; k < NPIX * NCH / 8; k += blockDim.x)
      reinterpret_cast<uint4*>(sdy)[k] =
          reinterpret_cast<const uint4*>(dY + (size_t)pp * NPIX * NCH)[k];
    __syncthreads();
    if (threadIdx.x < NCH)
      for (int px = 0; px < NPIX; ++px)
        dbs += __bfloat162float(sdy[px * NCH + threadIdx.x]);
    for (int ks = 0; ks < NPIX / 16; ++ks) {
      const int pb = ks * 16;
      unsigned a[4], b[4];
      ldsm_x4_t(a, sdy + (pb + (lane & 7) + 8 * (lane >> 4)) * NCH +
                       8 * ((lane >> 3) & 1));
      ldsm_x4_t(b, tap_row(tile, pb + (lane & 7) + 8 * ((lane >> 3) & 1), tap) +
                       8 * (lane >> 4));
      mma16816(acc[0], a, b[0], b[1]);
      mma16816(acc[1], a, b[2], b[3]);
    }
  }
#pragma unroll
  for (int nt = 0; nt < 2; ++nt)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int co = (lane >> 2) + 8 * h;
      const int ci = nt * 8 + (lane & 3) * 2;
      atomicAdd(&dW[co * KK + tap * 16 + ci], acc[nt][2 * h]);
      atomicAdd(&dW[co * KK + tap * 16 + ci + 1], acc[nt][2 * h + 1]);
    }
  if (threadIdx.x < NCH) atomicAdd(&db[threadIdx.x], dbs);
}

// Head: v = mean_p a3[p][:], logit = wh . v + bh.
__global__ void k_head(const bf16* __restrict__ a3, const float* __restrict__ wh,
                       const float* __restrict__ bh, float* __restrict__ logit,
                       float* __restrict__ vout, int npatch) {
  const int p = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (p >= npatch) return;
  const bf16* a = a3 + (size_t)p * NPIX * NCH;
  // lane handles channel lane % 16 over half of the pixels
  const int c = lane & 15, half = lane >> 4;
  float s = 0.f;
  for (int px = half; px < NPIX; px += 2) s += __bfloat162float(a[px * NCH + c]);
  s += __shfl_xor_sync(0xffffffffu, s, 16);
  const float v = s * (1.0f / NPIX);
  if (vout && lane < 16) vout[(size_t)p * NCH + c] = v;
  float z = lane < 16 ? wh[c] * v : 0.f;
  for (int o = 8; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
  if (lane == 0) logit[p] = z + bh[0];
}

// Head backward for binary cross-entropy on the logits: dlogit =
// w_y (sigmoid(z) - y) / n; dwh += dlogit v; dbh += dlogit;
// dA3[p][c] = dlogit wh[c] / 256 where a3 > 0 (relu), else 0.
__global__ void k_head_bwd(const float* __restrict__ logit,
                           const float* __restrict__ label,
                           const float* __restrict__ v,
                           const bf16* __restrict__ a3,
                           const float* __restrict__ wh, float pos_weight,
                           float inv_n, float* __restrict__ dwh,
                           float* __restrict__ dbh, bf16* __restrict__ dY3,
                           float* __restrict__ loss) {
  const int p = blockIdx.x;
  const float z = logit[p], y = label[p];
  const float sg = 1.f / (1.f + expf(-z));
  const float w = y > 0.5f ? pos_weight : 1.f;
  const float dz = w * (sg - y) * inv_n;
  if (threadIdx.x < NCH) atomicAdd(&dwh[threadIdx.x], dz * v[(size_t)p * NCH + threadIdx.x]);
  if (threadIdx.x == 0) {
    atomicAdd(dbh, dz);
    // softplus form of the cross-entropy
    const float l = fmaxf(z, 0.f) - z * y + log1pf(expf(-fabsf(z)));
    atomicAdd(loss, w * l * inv_n);
  }
  const bf16* a = a3 + (size_t)p * NPIX * NCH;
  bf16* d = dY3 + (size_t)p * NPIX * NCH;
  for (int k = threadIdx.x; k < NPIX * NCH; k += blockDim.x) {
    const int c = k & 15;
    const float g = __bfloat162float(a[k]) > 0.f ? dz * wh[c] * (1.0f / NPIX) : 0.f;
    d[k] = __float2bfloat16_rn(g);
  }
}

// Adam on the FP32 master parameters, then the BF16 copies of the conv
// weights and of their flipped transposes (the input-gradient pass):
// Wf[ci][(8 - tap)*16 + co] = W[co][tap*16 + ci].
__global__ void k_adam(float* __restrict__ prm, const float* __restrict__ grad,
                       float* __restrict__ m, float* __restrict__ v, int n,
                       float lr, float b1, float b2, float eps, float c1,
                       float c2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float g = grad[k];
  const float mk = b1 * m[k] + (1.f - b1) * g;
  const float vk = b2 * v[k] + (1.f - b2) * g * g;
  m[k] = mk;
  v[k] = vk;
  prm[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
}

__global__ void k_cast_weights(const float* __restrict__ prm, int layer_stride,
                               bf16* __restrict__ wb, bf16* __restrict__ wf) {
  const int l = blockIdx.y;
  const float* W = prm + (size_t)l * layer_stride;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= NCH * KK) return;
  const int co = k / KK, kk = k % KK, tap = kk / 16, ci = kk % 16;
  const bf16 w = __float2bfloat16_rn(W[k]);
  wb[(size_t)l * NCH * KK + k] = w;
  wf[(size_t)l * NCH * KK + ci * KK + (8 - tap) * 16 + co] = w;
}

__global__ void k_to_bf16(const float* __restrict__ x, bf16* __restrict__ y,
                          size_t n) {
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) y[k] = __float2bfloat16_rn(x[k]);
}

// Minibatch gather: xb[k] = x[idx[k]] (one CTA per sample), yb[k] = y[idx[k]].
__global__ void k_gather(const bf16* __restrict__ x, const float* __restrict__ y,
                         const int* __restrict__ idx, bf16* __restrict__ xb,
                         float* __restrict__ yb) {
  const int k = blockIdx.x;
  const int src = idx[k];
  const uint4* s4 = reinterpret_cast<const uint4*>(x + (size_t)src * NPAD * NCH);
  uint4* d4 = reinterpret_cast<uint4*>(xb + (size_t)k * NPAD * NCH);
  for (int t = threadIdx.x; t < NPAD * 2; t += blockDim.x) d4[t] = s4[t];
  if (threadIdx.x == 0) yb[k] = y[src];
}

inline int ok() { return cudaGetLastError() == cudaSuccess ? 0 : -2; }

}  // namespace

namespace gf {

// Parameter block (FP32): W1, b1, W2, b2, W3, b3 (stride 144*16 + 16 each),
// then wh[16], bh[1].
constexpr int CNN_LAYER = NCH * KK + NCH;
constexpr int CNN_NPARAM = 3 * CNN_LAYER + NCH + 1;

int cnn_nparam() { return CNN_NPARAM; }

// Forward pass of npatch feature tiles x0 (BF16) with the BF16 weights wb:
// fills a1, a2, a3, the pooled features v and the logits.
int cnn_forward(const void* x0, const void* wb, const float* prm, void* a1,
                void* a2, void* a3, float* v, float* logit, int npatch,
                void* stream) {
  if (npatch <= 0) return 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bf16* W = static_cast<const bf16*>(wb);
  k_conv<true, true, false, true><<<npatch, 256, 0, st>>>(
      static_cast<const bf16*>(x0), W, prm + NCH * KK, nullptr, static_cast<bf16*>(a1));
  k_conv<true, true, false, false><<<npatch, 256, 0, st>>>(
      static_cast<const bf16*>(a1), W + NCH * KK, prm + CNN_LAYER + NCH * KK, nullptr,
      static_cast<bf16*>(a2));
  k_conv<true, true, false, false><<<npatch, 256, 0, st>>>(
      static_cast<const bf16*>(a2), W + 2 * NCH * KK, prm + 2 * CNN_LAYER + NCH * KK,
      nullptr, static_cast<bf16*>(a3));
  k_head<<<(npatch + 7) / 8, 256, 0, st>>>(static_cast<const bf16*>(a3),
                                            prm + 3 * CNN_LAYER,
                                            prm + 3 * CNN_LAYER + NCH, logit, v,
                                            npatch);
  return ok();
}

// Backward pass after cnn_forward: accumulates the gradient of the mean
// weighted cross-entropy into grad (FP32, same layout as the parameters)
// and the loss into *loss.  d1, d2, d3 are BF16 scratch of the activations'
// shape.
int cnn_backward(const void* x0, const void* wf, const float* prm,
                 const void* a1, const void* a2, const void* a3, const float* v,
                 const float* logit, const float* label, float pos_weight,
                 float* grad, float* loss, void* d1, void* d2, void* d3,
                 int npatch, void* stream) {
  if (npatch <= 0) return 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bf16* Wf = static_cast<const bf16*>(wf);
  k_head_bwd<<<npatch, 256, 0, st>>>(logit, label, v, static_cast<const bf16*>(a3),
                                     prm + 3 * CNN_LAYER, pos_weight, 1.0f / npatch,
                                     grad + 3 * CNN_LAYER, grad + 3 * CNN_LAYER + NCH,
                                     static_cast<bf16*>(d3), loss);
  const int group = 8, blocks = (npatch + group - 1) / group;
  // layer 3: weight gradient from a2, input gradient through relu(a2)
  k_conv_dw<false><<<blocks, 288, 0, st>>>(static_cast<const bf16*>(d3),
                                    static_cast<const bf16*>(a2),
                                    grad + 2 * CNN_LAYER, grad + 2 * CNN_LAYER + NCH * KK,
                                    npatch, group);
  k_conv<false, false, true, false><<<npatch, 256, 0, st>>>(
      static_cast<const bf16*>(d3), Wf + 2 * NCH * KK, nullptr,
      static_cast<const bf16*>(a2), static_cast<bf16*>(d2));
  // layer 2
  k_conv_dw<false><<<blocks, 288, 0, st>>>(static_cast<const bf16*>(d2),
                                    static_cast<const bf16*>(a1),
                                    grad + CNN_LAYER, grad + CNN_LAYER + NCH * KK,
                                    npatch, group);
  k_conv<false, false, true, false><<<npatch, 256, 0, st>>>(
      static_cast<const bf16*>(d2), Wf + NCH * KK, nullptr,
      static_cast<const bf16*>(a1), static_cast<bf16*>(d1));
  // layer 1: weight gradient from the input features
  k_conv_dw<true><<<blocks, 288, 0, st>>>(static_cast<const bf16*>(d1),
                                    static_cast<const bf16*>(x0), grad,
                                    grad + NCH * KK, npatch, group);
  return ok();
}

int cnn_adam(float* prm, const float* grad, float* m, float* v, float lr,
             int t, void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const float b1 = 0.9f, b2 = 0.999f;
  float c1 = 1.f, c2 = 1.f;
  for (int k = 0; k < t; ++k) { c1 *= b1; c2 *= b2; }
  k_adam<<<(CNN_NPARAM + 255) / 256, 256, 0, st>>>(prm, grad, m, v, CNN_NPARAM, lr,
                                                   b1, b2, 1e-8f, 1.f - c1, 1.f - c2);
  return ok();
}

int cnn_cast(const float* prm, void* wb, void* wf, void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_cast_weights<<<dim3((NCH * KK + 255) / 256, 3), 256, 0, st>>>(
      prm, CNN_LAYER, static_cast<bf16*>(wb), static_cast<bf16*>(wf));
  return ok();
}

int cnn_gather(const void* x, const float* y, const int* idx, int n, void* xb,
               float* yb, void* stream) {
  if (n <= 0) return 0;
  k_gather<<<n, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      static_cast<const bf16*>(x), y, idx, static_cast<bf16*>(xb), yb);
  return ok();
}

int cnn_to_bf16(const float* x, void* y, size_t n, void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (n == 0) return 0;
  k_to_bf16<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, static_cast<bf16*>(y), n);
  return ok();
}

}  // namespace gf
