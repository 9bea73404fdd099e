// Weight-window importance network on the tensor cores: a 5 -> 64 -> 64 -> 64 -> 1 perceptron
// (tanh hidden units, linear output) mapping a phase-space point (x, y, z, group, t; each scaled
// to [-1, 1]) to log w_c, the log of the weight-window centre.  The paper's runs are analog or use
// implicit capture (its §3); the learned map is this library's variance-reduction extension.
//
// Every contraction runs on the tensor cores as BF16 x BF16 -> FP32 mma.sync m16n8k16: one warp
// owns a tile of 16 samples.  Forward activations stay in registers between layers (the FP32
// accumulator layout of two adjacent 8-column tiles is exactly the BF16 A-operand layout of the
// next layer's 16-wide K block); the backward pass stages activations per warp in shared memory
// to read the transposed operands of the weight gradients.  Parameters live as FP32 masters (Adam
// state, oracle layout) and BF16 copies for the MMAs, including transposed copies of W2 and W3.
//
// Parameter layout (FP32 masters, same order as the CPU oracle):
//   W1 [64][5], b1 [64], W2 [64][64], b2 [64], W3 [64][64], b3 [64], W4 [1][64], b4 [1].
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mcgb {
namespace mlp {

constexpr int H = 64;
constexpr int NIN = 5;
constexpr int O_W1 = 0, O_B1 = O_W1 + H * NIN, O_W2 = O_B1 + H, O_B2 = O_W2 + H * H, O_W3 = O_B2 + H,
              O_B3 = O_W3 + H * H, O_W4 = O_B3 + H, O_B4 = O_W4 + H, NPARAM = O_B4 + 1;
constexpr int LD = H + 8;  // padded row stride (bf16) of the staging tiles: conflict-light columns

// BF16 weights as the MMAs read them
struct __align__(16) Weights {
  __nv_bfloat16 w1[H * 16];   // [64][16], input K padded 5 -> 16 with zeros
  __nv_bfloat16 w2[H * H];    // [64][64] row = output neuron
  __nv_bfloat16 w3[H * H];
  __nv_bfloat16 w2t[H * H];   // transposed copies for the backward products dZ W
  __nv_bfloat16 w3t[H * H];
  __nv_bfloat16 w4[8 * H];    // [8][64], row 0 = W4, rows 1..7 zero (N padded 1 -> 8)
  float b1[H], b2[H], b3[H], w4f[H], b4;
};

// per-warp staging of a 16-sample tile for the backward pass
struct Stage {
  __nv_bfloat16 x[16 * 16];
  __nv_bfloat16 h1[16 * LD], h2[16 * LD], h3[16 * LD], dz[16 * LD];
};

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x (lower column) in the low half
  return *reinterpret_cast<const uint32_t*>(&v);
}
__device__ __forceinline__ uint32_t pack2b(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}
__device__ __forceinline__ uint32_t ld2(const __nv_bfloat16* p) {  // two consecutive bf16
  return *reinterpret_cast<const uint32_t*>(p);
}

// D = A (16x16 bf16, row) * B (16x8 bf16, col) + D (16x8 fp32)
__device__ __forceinline__ void mma(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// A fragment of K block kb from the accumulators of 8-column tiles 2kb and 2kb+1
__device__ __forceinline__ void afrag_from_acc(const float (*acc)[4], int kb, uint32_t a[4]) {
  a[0] = pack2(acc[2 * kb][0], acc[2 * kb][1]);
  a[1] = pack2(acc[2 * kb][2], acc[2 * kb][3]);
  a[2] = pack2(acc[2 * kb + 1][0], acc[2 * kb + 1][1]);
  a[3] = pack2(acc[2 * kb + 1][2], acc[2 * kb + 1][3]);
}

// out (16 x 64, as 8 accumulator tiles) = in (16 x 64 accumulators) * W^T + b, W row-major [64][64]
__device__ __forceinline__ void dense64(const float (*in)[4], const __nv_bfloat16* W, const float* b,
                                        float (*out)[4], int g, int t) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float b0 = b ? b[8 * j + 2 * t] : 0.f, b1 = b ? b[8 * j + 2 * t + 1] : 0.f;
    out[j][0] = b0;
    out[j][1] = b1;
    out[j][2] = b0;
    out[j][3] = b1;
  }
#pragma unroll
  for (int kb = 0; kb < 4; ++kb) {
    uint32_t a[4];
    afrag_from_acc(in, kb, a);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const __nv_bfloat16* row = W + (8 * j + g) * H + 16 * kb + 2 * t;
      mma(out[j], a, ld2(row), ld2(row + 8));
    }
  }
}

__device__ __forceinline__ void tanh_acc(float (*a)[4]) {
#pragma unroll
  for (int j = 0; j < 8; ++j)
#pragma unroll
    for (int e = 0; e < 4; ++e) a[j][e] = tanhf(a[j][e]);
}

// Forward pass of the 16 samples starting at r0 (rows >= n read as zeros).  h1..h3 receive the
// hidden activations; the return value of lanes with t == 0 is y for rows g and g+8 (in y[0], y[1]).
__device__ __forceinline__ void forward_tile(const Weights& W, const float* x, int n, int r0, float (*h1)[4],
                                             float (*h2)[4], float (*h3)[4], float y[2]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  // layer 1: A = x tile with K padded to 16 (only columns 0..4 are non-zero)
  auto xin = [&](int r, int c) -> float {
    return (r0 + r < n && c < NIN) ? x[(size_t)(r0 + r) * NIN + c] : 0.f;
  };
  uint32_t a[4];
  a[0] = pack2(xin(g, 2 * t), xin(g, 2 * t + 1));
  a[1] = pack2(xin(g + 8, 2 * t), xin(g + 8, 2 * t + 1));
  a[2] = 0u;
  a[3] = 0u;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float b0 = W.b1[8 * j + 2 * t], b1 = W.b1[8 * j + 2 * t + 1];
    h1[j][0] = b0;
    h1[j][1] = b1;
    h1[j][2] = b0;
    h1[j][3] = b1;
    const __nv_bfloat16* row = W.w1 + (8 * j + g) * 16 + 2 * t;
    mma(h1[j], a, ld2(row), ld2(row + 8));
  }
  tanh_acc(h1);
  dense64(h1, W.w2, W.b2, h2, g, t);
  tanh_acc(h2);
  dense64(h2, W.w3, W.b3, h3, g, t);
  tanh_acc(h3);
  // layer 4: one 8-column tile, only column 0 is real
  float o[4] = {W.b4, W.b4, W.b4, W.b4};
#pragma unroll
  for (int kb = 0; kb < 4; ++kb) {
    afrag_from_acc(h3, kb, a);
    const __nv_bfloat16* row = W.w4 + g * H + 16 * kb + 2 * t;
    mma(o, a, ld2(row), ld2(row + 8));
  }
  y[0] = o[0];
  y[1] = o[2];
}


// stage a 16 x 64 accumulator tile (C layout) as bf16 rows [r][LD]
__device__ __forceinline__ void stage_acc(__nv_bfloat16* dst, const float (*acc)[4], int g, int t) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    *reinterpret_cast<uint32_t*>(dst + g * LD + 8 * j + 2 * t) = pack2(acc[j][0], acc[j][1]);
    *reinterpret_cast<uint32_t*>(dst + (g + 8) * LD + 8 * j + 2 * t) = pack2(acc[j][2], acc[j][3]);
  }
}

// sum over the 8 row groups (lanes with equal t) of a warp
__device__ __forceinline__ float sum_over_g(float v) {
  v += __shfl_xor_sync(0xFFFFFFFFu, v, 4);
  v += __shfl_xor_sync(0xFFFFFFFFu, v, 8);
  v += __shfl_xor_sync(0xFFFFFFFFu, v, 16);
  return v;
}

// bias gradient of a layer: sum over the tile's rows of dz (accumulator layout)
__device__ __forceinline__ void bias_grad(float* gb, const float (*dz)[4], int g, int t) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float s0 = sum_over_g(dz[j][0] + dz[j][2]);
    const float s1 = sum_over_g(dz[j][1] + dz[j][3]);
    if (g == 0) {
      atomicAdd(gb + 8 * j + 2 * t, s0);
      atomicAdd(gb + 8 * j + 2 * t + 1, s1);
    }
  }
}

// weight gradient dW[j][k] += sum_r dz[r][j] * a[r][k]: (dz^T, 64 x 16) x (a, 16 x ncol), read
// transposed from the staged tiles; ncol = 64 (hidden inputs) or 5 (network inputs, staged 16 wide)
__device__ __forceinline__ void weight_grad(float* gW, const __nv_bfloat16* dz, const __nv_bfloat16* a, int lda,
                                            int ncol, int g, int t) {
  const int ntile = ncol > 8 ? ncol / 8 : 1;
  for (int mj = 0; mj < 4; ++mj) {
    const int j0 = 16 * mj + g;
    uint32_t af[4];
    af[0] = pack2b(dz[(2 * t) * LD + j0], dz[(2 * t + 1) * LD + j0]);
    af[1] = pack2b(dz[(2 * t) * LD + j0 + 8], dz[(2 * t + 1) * LD + j0 + 8]);
    af[2] = pack2b(dz[(2 * t + 8) * LD + j0], dz[(2 * t + 9) * LD + j0]);
    af[3] = pack2b(dz[(2 * t + 8) * LD + j0 + 8], dz[(2 * t + 9) * LD + j0 + 8]);
    for (int nk = 0; nk < ntile; ++nk) {
      const int k0 = 8 * nk + g;
      const uint32_t b0 = pack2b(a[(2 * t) * lda + k0], a[(2 * t + 1) * lda + k0]);
      const uint32_t b1 = pack2b(a[(2 * t + 8) * lda + k0], a[(2 * t + 9) * lda + k0]);
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      mma(c, af, b0, b1);
      const int k = 8 * nk + 2 * t;
      if (k < ncol) {
        atomicAdd(gW + j0 * ncol + k, c[0]);
        atomicAdd(gW + (j0 + 8) * ncol + k, c[2]);
      }
      if (k + 1 < ncol) {
        atomicAdd(gW + j0 * ncol + k + 1, c[1]);
        atomicAdd(gW + (j0 + 8) * ncol + k + 1, c[3]);
      }
    }
  }
}

// Forward and backward pass of the 16 samples at r0 for the loss
//   L = (1/n) sum_r wt[r] (y[r] - target[r])^2,
// adding dL/dparams into gsm[NPARAM] (shared) and the tile's loss into *loss (per-thread part).
__device__ void tile_loss_grad(const Weights& W, Stage& S, const float* x, const float* tgt, const float* wt, int n,
                               int r0, float inv_n, float* gsm, float* loss) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  float h1[8][4], h2[8][4], h3[8][4], y[2];
  forward_tile(W, x, n, r0, h1, h2, h3, y);
  // output error, rows g and g+8 (computed on lanes t == 0, broadcast to the row group)
  float dy0 = 0.f, dy1 = 0.f;
  if (t == 0) {
    if (r0 + g < n) {
      const float e = y[0] - tgt[r0 + g], w = wt ? wt[r0 + g] : 1.f;
      dy0 = 2.f * w * e * inv_n;
      *loss += w * e * e * inv_n;
    }
    if (r0 + g + 8 < n) {
      const float e = y[1] - tgt[r0 + g + 8], w = wt ? wt[r0 + g + 8] : 1.f;
      dy1 = 2.f * w * e * inv_n;
      *loss += w * e * e * inv_n;
    }
  }
  dy0 = __shfl_sync(0xFFFFFFFFu, dy0, lane & ~3);
  dy1 = __shfl_sync(0xFFFFFFFFu, dy1, lane & ~3);
  {
    const float s = sum_over_g(t == 0 ? dy0 + dy1 : 0.f);
    if (lane == 0) atomicAdd(gsm + O_B4, s);
  }
  // dW4 and dz3 = dy W4 (1 - h3^2)
  float dz[8][4];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int c = 8 * j + 2 * t;
    const float s0 = sum_over_g(dy0 * h3[j][0] + dy1 * h3[j][2]);
    const float s1 = sum_over_g(dy0 * h3[j][1] + dy1 * h3[j][3]);
    if (g == 0) {
      atomicAdd(gsm + O_W4 + c, s0);
      atomicAdd(gsm + O_W4 + c + 1, s1);
    }
    dz[j][0] = dy0 * W.w4f[c] * (1.f - h3[j][0] * h3[j][0]);
    dz[j][1] = dy0 * W.w4f[c + 1] * (1.f - h3[j][1] * h3[j][1]);
    dz[j][2] = dy1 * W.w4f[c] * (1.f - h3[j][2] * h3[j][2]);
    dz[j][3] = dy1 * W.w4f[c + 1] * (1.f - h3[j][3] * h3[j][3]);
  }
  // layer 3
  stage_acc(S.dz, dz, g, t);
  stage_acc(S.h2, h2, g, t);
  __syncwarp();
  weight_grad(gsm + O_W3, S.dz, S.h2, LD, H, g, t);
  bias_grad(gsm + O_B3, dz, g, t);
  float dh[8][4];
  dense64(dz, W.w3t, nullptr, dh, g, t);
#pragma unroll
  for (int j = 0; j < 8; ++j)
#pragma unroll
    for (int e = 0; e < 4; ++e) dz[j][e] = dh[j][e] * (1.f - h2[j][e] * h2[j][e]);
  // layer 2
  __syncwarp();
  stage_acc(S.dz, dz, g, t);
  stage_acc(S.h1, h1, g, t);
  __syncwarp();
  weight_grad(gsm + O_W2, S.dz, S.h1, LD, H, g, t);
  bias_grad(gsm + O_B2, dz, g, t);
  dense64(dz, W.w2t, nullptr, dh, g, t);
#pragma unroll
  for (int j = 0; j < 8; ++j)
#pragma unroll
    for (int e = 0; e < 4; ++e) dz[j][e] = dh[j][e] * (1.f - h1[j][e] * h1[j][e]);
  // layer 1: inputs staged as a 16 x 16 tile (columns >= 5 zero)
  __syncwarp();
  stage_acc(S.dz, dz, g, t);
  for (int i = lane; i < 256; i += 32) {
    const int r = i >> 4, c = i & 15;
    S.x[i] = __float2bfloat16_rn((r0 + r < n && c < NIN) ? x[(size_t)(r0 + r) * NIN + c] : 0.f);
  }
  __syncwarp();
  weight_grad(gsm + O_W1, S.dz, S.x, 16, NIN, g, t);
  bias_grad(gsm + O_B1, dz, g, t);
  __syncwarp();
}

// BF16 copies of one master parameter
__device__ __forceinline__ void scatter_param(Weights& W, int i, float v) {
  const __nv_bfloat16 b = __float2bfloat16_rn(v);
  if (i < O_B1) {
    W.w1[(i / NIN) * 16 + (i % NIN)] = b;
  } else if (i < O_W2) {
    W.b1[i - O_B1] = v;
  } else if (i < O_B2) {
    const int j = (i - O_W2) / H, k = (i - O_W2) % H;
    W.w2[j * H + k] = b;
    W.w2t[k * H + j] = b;
  } else if (i < O_W3) {
    W.b2[i - O_B2] = v;
  } else if (i < O_B3) {
    const int j = (i - O_W3) / H, k = (i - O_W3) % H;
    W.w3[j * H + k] = b;
    W.w3t[k * H + j] = b;
  } else if (i < O_W4) {
    W.b3[i - O_B3] = v;
  } else if (i < O_B4) {
    W.w4[i - O_W4] = b;
    W.w4f[i - O_W4] = v;
  } else {
    W.b4 = v;
  }
}

// zero the padding of the BF16 copies (input columns 5..15, output rows 1..7)
__device__ __forceinline__ void clear_padding(Weights& W) {
  for (int i = threadIdx.x; i < H * 16; i += blockDim.x)
    if ((i & 15) >= NIN) W.w1[i] = __float2bfloat16_rn(0.f);
  for (int i = H + threadIdx.x; i < 8 * H; i += blockDim.x) W.w4[i] = __float2bfloat16_rn(0.f);
}

__global__ void k_refresh(const float* master, Weights* W) {
  clear_padding(*W);
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) scatter_param(*W, i, master[i]);
}

__device__ __forceinline__ void load_weights(Weights& dst, const Weights* src) {
  const uint4* s = reinterpret_cast<const uint4*>(src);
  uint4* d = reinterpret_cast<uint4*>(&dst);
  for (int i = threadIdx.x; i < (int)(sizeof(Weights) / 16); i += blockDim.x) d[i] = s[i];
  __syncthreads();
}

__global__ void k_forward(const Weights* Wg, const float* x, float* y, int n) {
  extern __shared__ __align__(16) unsigned char sm[];
  Weights& W = *reinterpret_cast<Weights*>(sm);
  load_weights(W, Wg);
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int warps = gridDim.x * (blockDim.x >> 5);
  for (int tile = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); tile * 16 < n; tile += warps) {
    float h1[8][4], h2[8][4], h3[8][4], out[2];
    forward_tile(W, x, n, tile * 16, h1, h2, h3, out);
    if (t == 0) {
      if (tile * 16 + g < n) y[tile * 16 + g] = out[0];
      if (tile * 16 + g + 8 < n) y[tile * 16 + g + 8] = out[1];
    }
  }
}

// dynamic shared memory of the gradient kernels: [Weights][gradients NPARAM floats][Stage per warp]
__host__ __device__ constexpr size_t grad_smem(int warps) {
  return ((sizeof(Weights) + 15) / 16) * 16 + ((NPARAM * 4 + 15) / 16) * 16 + (size_t)warps * sizeof(Stage);
}

__global__ void k_loss_grad(const Weights* Wg, const float* x, const float* tgt, const float* wt, int n,
                            float* grad, float* loss) {
  extern __shared__ __align__(16) unsigned char sm[];
  Weights& W = *reinterpret_cast<Weights*>(sm);
  float* gsm = reinterpret_cast<float*>(sm + ((sizeof(Weights) + 15) / 16) * 16);
  Stage* st = reinterpret_cast<Stage*>(reinterpret_cast<unsigned char*>(gsm) + ((NPARAM * 4 + 15) / 16) * 16);
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) gsm[i] = 0.f;
  load_weights(W, Wg);
  const int warp = threadIdx.x >> 5, warps = gridDim.x * (blockDim.x >> 5);
  float l = 0.f;
  for (int tile = blockIdx.x * (blockDim.x >> 5) + warp; tile * 16 < n; tile += warps)
    tile_loss_grad(W, st[warp], x, tgt, wt, n, tile * 16, 1.f / (float)n, gsm, &l);
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xFFFFFFFFu, l, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, l);
  __syncthreads();
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) atomicAdd(grad + i, gsm[i]);
}

// Grid barrier of the training kernel (a cooperative launch, every CTA resident): the wait is
// bounded; on expiry the CTA records an error, and every CTA leaves the epoch loop at its next
// barrier, so that a stuck barrier ends the kernel instead of hanging it.
struct TrainSync {
  unsigned int count, gen;
  int err, pad;
  float loss[2];  // loss of the even / odd epochs
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ bool train_grid_sync(TrainSync* s) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned gen = ld_acquire_u32(&s->gen);
    __threadfence();
    if (atomicAdd(&s->count, 1u) == gridDim.x - 1) {
      atomicExch(&s->count, 0u);
      __threadfence();
      atomicAdd(&s->gen, 1u);
    } else {
      unsigned long long polls = 0;
      while (ld_acquire_u32(&s->gen) == gen) {
        if (*(volatile int*)&s->err) break;
        if (++polls > (1ull << 26)) {
          atomicExch(&s->err, 1);
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    s_ok = *(volatile int*)&s->err == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

// the BF16 weights from global memory through L2 (other CTAs rewrite them between epochs)
__device__ __forceinline__ void load_weights_cg(Weights& dst, const Weights* src) {
  const uint4* s = reinterpret_cast<const uint4*>(src);
  uint4* d = reinterpret_cast<uint4*>(&dst);
  for (int i = threadIdx.x; i < (int)(sizeof(Weights) / 16); i += blockDim.x) d[i] = __ldcg(s + i);
  __syncthreads();
}

// Full-batch Adam over a grid of CTAs (one cooperative launch for all epochs).  Every epoch each
// warp of the grid computes the loss gradient of its 16-sample tiles on the tensor cores into its
// CTA's shared gradient; the CTAs add theirs into the epoch's global gradient; after a grid
// barrier each CTA updates its share of the FP32 masters with Adam and writes their BF16 copies;
// after a second barrier every CTA reloads the BF16 weights.  The gradients of even and odd epochs
// alternate between two buffers, each zeroed an epoch ahead, so two barriers per epoch suffice.
__global__ void k_train(float* master, float* m1, float* m2, Weights* Wg, const float* x, const float* tgt,
                        const float* wt, int n, int epochs, float lr, long long step0, float* last_loss, float* gbuf,
                        TrainSync* sync) {
  extern __shared__ __align__(16) unsigned char sm[];
  Weights& W = *reinterpret_cast<Weights*>(sm);
  float* gsm = reinterpret_cast<float*>(sm + ((sizeof(Weights) + 15) / 16) * 16);
  Stage* st = reinterpret_cast<Stage*>(reinterpret_cast<unsigned char*>(gsm) + ((NPARAM * 4 + 15) / 16) * 16);
  load_weights_cg(W, Wg);
  const int warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int gw = blockIdx.x * wpb + warp, nw = gridDim.x * wpb;
  const int chunk = (NPARAM + gridDim.x - 1) / gridDim.x;
  const int p0 = blockIdx.x * chunk, p1 = p0 + chunk < NPARAM ? p0 + chunk : NPARAM;
  const float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
  bool ok = true;
  int e = 0;
  for (; e < epochs && ok; ++e) {
    float* gcur = gbuf + (e & 1) * NPARAM;
    float* gnext = gbuf + ((e + 1) & 1) * NPARAM;
    for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) gsm[i] = 0.f;
    __syncthreads();
    float l = 0.f;
    for (int tile = gw; tile * 16 < n; tile += nw)
      tile_loss_grad(W, st[warp], x, tgt, wt, n, tile * 16, 1.f / (float)n, gsm, &l);
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xFFFFFFFFu, l, o);
    if ((threadIdx.x & 31) == 0 && l != 0.f) atomicAdd(&sync->loss[e & 1], l);
    __syncthreads();
    for (int i = threadIdx.x; i < NPARAM; i += blockDim.x)
      if (gsm[i] != 0.f) atomicAdd(gcur + i, gsm[i]);
    if (!(ok = train_grid_sync(sync))) break;
    const float step = (float)(step0 + e + 1);
    const float c1 = 1.f - powf(beta1, step), c2 = 1.f - powf(beta2, step);
    for (int i = p0 + threadIdx.x; i < p1; i += blockDim.x) {
      const float gr = __ldcg(gcur + i);
      const float a = beta1 * m1[i] + (1.f - beta1) * gr;
      const float b = beta2 * m2[i] + (1.f - beta2) * gr * gr;
      m1[i] = a;
      m2[i] = b;
      const float p = master[i] - lr * (a / c1) / (sqrtf(b / c2) + eps);
      master[i] = p;
      scatter_param(*Wg, i, p);
      gnext[i] = 0.f;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) sync->loss[(e + 1) & 1] = 0.f;
    if (!(ok = train_grid_sync(sync))) break;
    load_weights_cg(W, Wg);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && last_loss)
    *last_loss = epochs == 0 ? 0.f : (ok ? *(volatile float*)&sync->loss[(epochs - 1) & 1] : __int_as_float(0x7FC00000));
}

// window centres from the network: centre[i] = ref * exp(scale * y[i]), y clamped to [ymin, ymax]
__global__ void k_centres(const float* y, int n, double scale, double ymin, double ymax, double ref, double* centre) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double v = scale * (double)y[i];
    v = v < ymin ? ymin : (v > ymax ? ymax : v);
    centre[i] = ref * exp(v);
  }
}

}  // namespace mlp

// ------------------------------------------------------------------------------------------ launchers
size_t mlp_param_count() { return mlp::NPARAM; }
size_t mlp_weights_bytes() { return sizeof(mlp::Weights); }

cudaError_t mlp_refresh(const float* master, void* Wg, cudaStream_t s) {
  mlp::k_refresh<<<1, 256, 0, s>>>(master, reinterpret_cast<mlp::Weights*>(Wg));
  return cudaGetLastError();
}

cudaError_t mlp_forward(const void* Wg, const float* x, float* y, int n, cudaStream_t s) {
  const size_t smem = sizeof(mlp::Weights);
  cudaError_t e = cudaFuncSetAttribute(mlp::k_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int tiles = (n + 15) / 16;
  int grid = (tiles + 7) / 8;
  if (grid > 152 * 4) grid = 152 * 4;
  if (grid < 1) grid = 1;
  mlp::k_forward<<<grid, 256, smem, s>>>(reinterpret_cast<const mlp::Weights*>(Wg), x, y, n);
  return cudaGetLastError();
}

cudaError_t mlp_loss_grad(const void* Wg, const float* x, const float* tgt, const float* wt, int n, float* grad,
                          float* loss, cudaStream_t s) {
  const size_t smem = mlp::grad_smem(8);
  cudaError_t e = cudaFuncSetAttribute(mlp::k_loss_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int tiles = (n + 15) / 16;
  int grid = (tiles + 7) / 8;
  if (grid > 152) grid = 152;
  if (grid < 1) grid = 1;
  mlp::k_loss_grad<<<grid, 256, smem, s>>>(reinterpret_cast<const mlp::Weights*>(Wg), x, tgt, wt, n, grad, loss);
  return cudaGetLastError();
}

size_t mlp_train_scratch_bytes() { return 2 * mlp::NPARAM * 4 + sizeof(mlp::TrainSync); }

cudaError_t mlp_train(float* master, float* m1, float* m2, void* Wg, const float* x, const float* tgt, const float* wt,
                      int n, int epochs, float lr, long long step0, float* last_loss, void* scratch, cudaStream_t s) {
  const size_t smem = mlp::grad_smem(8);
  cudaError_t e = cudaFuncSetAttribute(mlp::k_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // one warp per 16-sample tile where the SMs allow (one CTA of 8 warps per SM), cooperative
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mlp::k_train, 256, smem)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int tiles = (n + 15) / 16;
  int grid = (tiles + 7) / 8;
  if (grid > sms * per_sm) grid = sms * per_sm;
  if (grid < 1) grid = 1;
  float* gbuf = reinterpret_cast<float*>(scratch);
  mlp::TrainSync* sync = reinterpret_cast<mlp::TrainSync*>(gbuf + 2 * mlp::NPARAM);
  if ((e = cudaMemsetAsync(scratch, 0, mlp_train_scratch_bytes(), s)) != cudaSuccess) return e;
  mlp::Weights* W = reinterpret_cast<mlp::Weights*>(Wg);
  void* args[] = {&master, &m1, &m2, &W, const_cast<float**>(&x), const_cast<float**>(&tgt), const_cast<float**>(&wt),
                  &n, &epochs, &lr, &step0, &last_loss, &gbuf, &sync};
  e = cudaLaunchCooperativeKernel((const void*)mlp::k_train, grid, 256, args, smem, s);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t mlp_centres(const float* y, int n, double scale, double ymin, double ymax, double ref, double* centre,
                        cudaStream_t s) {
  int grid = (n + 255) / 256;
  if (grid > 1024) grid = 1024;
  if (grid < 1) grid = 1;
  mlp::k_centres<<<grid, 256, 0, s>>>(y, n, scale, ymin, ymax, ref, centre);
  return cudaGetLastError();
}

}  // namespace mcgb
