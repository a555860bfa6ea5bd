// Kernels of the learned warm start: a small 3-D U-Net that maps a target
// specification to an initial density for the optimizer. Not part of the paper
// (the paper's optimizer starts from rho = 1); the optimizer always refines the
// network's output, so the network only changes how many steps are needed.
//
// Layouts: activations channels-last [N][D][H][W][C], C a multiple of 16 (padded
// channels are zero); bfloat16 activations, float32 activation gradients.
// Weights: float32 master [27][Cin][Cout] (tap = (dz+1)*9 + (dy+1)*3 + (dx+1));
// bfloat16 copies Wf [27][Cout][Cin] (forward) and Wb [27][Cin][Cout] (backward).
// 3x3x3 convolutions (stride 1, zero padding 1) forward and backward-data are
// implicit GEMMs on the tensor cores (mma m16n8k16, bfloat16 in, float32
// accumulate); so are the weight gradients (a GEMM over voxels per tap, the output
// gradient rounded to bfloat16 as in the data gradient).
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/topomag_net.h"

namespace {

using bf16 = __nv_bfloat16;

__device__ __forceinline__ uint32_t pack2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

__device__ __forceinline__ void mma16816(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

struct Vox {
  int n, z, y, x;
};
__device__ __forceinline__ Vox vox_of(long long v, int D, int H, int W) {
  Vox r;
  r.x = (int)(v % W);
  long long t = v / W;
  r.y = (int)(t % H);
  t /= H;
  r.z = (int)(t % D);
  r.n = (int)(t / D);
  return r;
}

constexpr int MT = 2;        // 16-voxel m tiles per warp
constexpr int WARPS = 4;     // warps per block
constexpr int VB = 16 * MT * WARPS;  // voxels per block

// Forward (MODE 0): out[v][co] = act(sum_{tap,ci} in[v + off][ci] Wf[tap][co][ci] + b[co])
// Backward data (MODE 1): din[v][ci] = sum_{tap,co} dout[v - off][co] Wb[tap][ci][co]
// KC = input channels of the GEMM (Cin fwd, Cout bwd); NO = output channels (<= 64).
template <int MODE, int NO>
__global__ void __launch_bounds__(WARPS * 32) k_conv_mma(const void* src, const bf16* Wt, const float* bias, void* dst,
                                                         int N, int D, int H, int W, int KC, int relu) {
  constexpr int NT = NO / 8;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const long long nvox = (long long)N * D * H * W;
  const long long v0 = (long long)blockIdx.x * VB + warp * 16 * MT;
  Vox rv[MT][2];
  bool rok[MT][2];
#pragma unroll
  for (int m = 0; m < MT; m++)
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const long long v = v0 + m * 16 + g + 8 * h;
      rok[m][h] = v < nvox;
      rv[m][h] = vox_of(rok[m][h] ? v : 0, D, H, W);
    }
  float acc[MT][NT][4];
#pragma unroll
  for (int m = 0; m < MT; m++)
#pragma unroll
    for (int j = 0; j < NT; j++)
#pragma unroll
      for (int q = 0; q < 4; q++) acc[m][j][q] = 0.0f;

  for (int tap = 0; tap < 27; tap++) {
    int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
    if (MODE == 1) {
      dz = -dz;
      dy = -dy;
      dx = -dx;
    }
    long long base[MT][2];
#pragma unroll
    for (int m = 0; m < MT; m++)
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const Vox& q = rv[m][h];
        const int z = q.z + dz, y = q.y + dy, x = q.x + dx;
        const bool in = rok[m][h] && z >= 0 && z < D && y >= 0 && y < H && x >= 0 && x < W;
        base[m][h] = in ? ((((long long)q.n * D + z) * H + y) * W + x) * KC : -1;
      }
    for (int k0 = 0; k0 < KC; k0 += 16) {
      uint32_t a[MT][4];
#pragma unroll
      for (int m = 0; m < MT; m++)
#pragma unroll
        for (int r = 0; r < 4; r++) {
          const int h = r & 1, col = k0 + 2 * t + 8 * (r >> 1);
          const long long b = base[m][h];
          if (b < 0) {
            a[m][r] = 0u;
          } else if (MODE == 0) {
            a[m][r] = *reinterpret_cast<const uint32_t*>(reinterpret_cast<const bf16*>(src) + b + col);
          } else {
            const float2 f = *reinterpret_cast<const float2*>(reinterpret_cast<const float*>(src) + b + col);
            a[m][r] = pack2(f.x, f.y);
          }
        }
#pragma unroll
      for (int j = 0; j < NT; j++) {
        // Wt[tap][n][k] with k (the reduced channel) contiguous
        const bf16* wr = Wt + ((long long)tap * NO + j * 8 + g) * KC + k0 + 2 * t;
        uint32_t b[2];
        b[0] = *reinterpret_cast<const uint32_t*>(wr);
        b[1] = *reinterpret_cast<const uint32_t*>(wr + 8);
#pragma unroll
        for (int m = 0; m < MT; m++) mma16816(acc[m][j], a[m], b);
      }
    }
  }
  // epilogue: rows g (c0, c1) and g + 8 (c2, c3), columns j*8 + 2t, +1
#pragma unroll
  for (int m = 0; m < MT; m++)
#pragma unroll
    for (int h = 0; h < 2; h++) {
      if (!rok[m][h]) continue;
      const long long v = v0 + m * 16 + g + 8 * h;
#pragma unroll
      for (int j = 0; j < NT; j++) {
        const int col = j * 8 + 2 * t;
        float o0 = acc[m][j][2 * h], o1 = acc[m][j][2 * h + 1];
        if (MODE == 0) {
          if (bias) {
            o0 += bias[col];
            o1 += bias[col + 1];
          }
          if (relu) {
            o0 = fmaxf(o0, 0.0f);
            o1 = fmaxf(o1, 0.0f);
          }
          *reinterpret_cast<uint32_t*>(reinterpret_cast<bf16*>(dst) + v * NO + col) = pack2(o0, o1);
        } else {
          float* d = reinterpret_cast<float*>(dst) + v * NO + col;
          if (relu) {  // accumulate into an existing gradient
            d[0] += o0;
            d[1] += o1;
          } else {
            d[0] = o0;
            d[1] = o1;
          }
        }
      }
    }
}

// dW[tap][ci][co] partial over a voxel range on the tensor cores: for one tap and one
// 16-channel tile of ci, dW_tile = sum_v in[v + off][ci] dout[v][co] is a 16 x Cout x
// (voxels) GEMM. Each step stages 64 voxels (shifted input rows, bfloat16; dout rows
// rounded to bfloat16) in shared memory; warp w takes voxels 16w..16w+15 as the k
// dimension of one m16n8k16 per 8 columns of co. The four warps' float32 sums are added
// in a fixed order into one partial per block.
constexpr int WVD = 64;  // voxels per staging step
template <int NT>
__global__ void __launch_bounds__(128) k_conv_dw_mma(const bf16* in, const float* dout, float* part, int N, int D,
                                                     int H, int W, int Cin, int Cout, int chunks_per_block) {
  constexpr int CO = NT * 8;
  __shared__ __align__(16) bf16 sa[WVD][16 + 8];
  __shared__ __align__(16) bf16 sb[WVD][CO + 8];
  __shared__ long long srow[WVD];
  __shared__ float red[4][16][CO];
  const int tap = blockIdx.y, mt = blockIdx.z;
  const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const long long nvox = (long long)N * D * H * W;
  float acc[NT][4];
#pragma unroll
  for (int j = 0; j < NT; j++)
#pragma unroll
    for (int q = 0; q < 4; q++) acc[j][q] = 0.0f;
  const long long vstart = (long long)blockIdx.x * chunks_per_block * WVD;
  for (int cidx = 0; cidx < chunks_per_block; cidx++) {
    const long long vb = vstart + (long long)cidx * WVD;
    if (vb >= nvox) break;
    __syncthreads();
    if (threadIdx.x < WVD) {  // source row of each staged voxel (-1: outside the grid)
      const long long v = vb + threadIdx.x;
      long long src = -1;
      if (v < nvox) {
        const Vox q = vox_of(v, D, H, W);
        const int z = q.z + dz, y = q.y + dy, x = q.x + dx;
        if (z >= 0 && z < D && y >= 0 && y < H && x >= 0 && x < W) src = (((long long)q.n * D + z) * H + y) * W + x;
      }
      srow[threadIdx.x] = src;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < WVD * 16; i += 128) {
      const int r = i >> 4, ci = i & 15;
      const long long src = srow[r];
      sa[r][ci] = src >= 0 ? in[src * Cin + mt * 16 + ci] : __float2bfloat16(0.0f);
    }
    for (int i = threadIdx.x; i < WVD * CO; i += 128) {
      const int r = i / CO, co = i - r * CO;
      const long long v = vb + r;
      sb[r][co] = __float2bfloat16(v < nvox ? dout[v * Cout + co] : 0.0f);
    }
    __syncthreads();
    const int k0 = warp * 16;
    uint32_t af[4];
    af[0] = (uint32_t)__bfloat16_as_ushort(sa[k0 + 2 * t][g]) | ((uint32_t)__bfloat16_as_ushort(sa[k0 + 2 * t + 1][g]) << 16);
    af[1] = (uint32_t)__bfloat16_as_ushort(sa[k0 + 2 * t][g + 8]) |
            ((uint32_t)__bfloat16_as_ushort(sa[k0 + 2 * t + 1][g + 8]) << 16);
    af[2] = (uint32_t)__bfloat16_as_ushort(sa[k0 + 2 * t + 8][g]) |
            ((uint32_t)__bfloat16_as_ushort(sa[k0 + 2 * t + 9][g]) << 16);
    af[3] = (uint32_t)__bfloat16_as_ushort(sa[k0 + 2 * t + 8][g + 8]) |
            ((uint32_t)__bfloat16_as_ushort(sa[k0 + 2 * t + 9][g + 8]) << 16);
#pragma unroll
    for (int j = 0; j < NT; j++) {
      const int n = j * 8 + g;
      uint32_t bfr[2];
      bfr[0] = (uint32_t)__bfloat16_as_ushort(sb[k0 + 2 * t][n]) | ((uint32_t)__bfloat16_as_ushort(sb[k0 + 2 * t + 1][n]) << 16);
      bfr[1] = (uint32_t)__bfloat16_as_ushort(sb[k0 + 2 * t + 8][n]) |
               ((uint32_t)__bfloat16_as_ushort(sb[k0 + 2 * t + 9][n]) << 16);
      mma16816(acc[j], af, bfr);
    }
  }
  // rows g (c0, c1) and g + 8 (c2, c3) of the tile, columns j*8 + 2t, +1
#pragma unroll
  for (int j = 0; j < NT; j++) {
    red[warp][g][j * 8 + 2 * t] = acc[j][0];
    red[warp][g][j * 8 + 2 * t + 1] = acc[j][1];
    red[warp][g + 8][j * 8 + 2 * t] = acc[j][2];
    red[warp][g + 8][j * 8 + 2 * t + 1] = acc[j][3];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 16 * CO; i += 128) {
    const int r = i / CO, co = i - r * CO;
    const float v = ((red[0][r][co] + red[1][r][co]) + red[2][r][co]) + red[3][r][co];
    part[((long long)blockIdx.x * 27 + tap) * Cin * Cout + (long long)(mt * 16 + r) * Cout + co] = v;
  }
}

// sum of the block partials in a fixed order; also the bias gradient
__global__ void k_dw_reduce(const float* part, int nblk, long long n, float* dW) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int b = 0; b < nblk; b++) s += part[(long long)b * n + i];
    dW[i] = s;
  }
}
__global__ void k_db(const float* dout, long long nvox, int C, float* db) {
  const int c = blockIdx.x;
  __shared__ float red[256];
  float s = 0.0f;
  for (long long v = threadIdx.x; v < nvox; v += blockDim.x) s += dout[v * C + c];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) db[c] = red[0];
}

// g *= (act > 0): ReLU backward through the stored bfloat16 activation
__global__ void k_relu_bwd(float* g, const bf16* act, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    if (!(__bfloat162float(act[i]) > 0.0f)) g[i] = 0.0f;
}

// 2x2x2 average pooling and its adjoint
__global__ void k_pool(const bf16* in, bf16* out, int N, int D, int H, int W, int C) {
  const long long n = (long long)N * (D / 2) * (H / 2) * (W / 2) * C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const Vox q = vox_of(i / C, D / 2, H / 2, W / 2);
    float s = 0.0f;
    for (int a = 0; a < 8; a++) {
      const int z = 2 * q.z + (a >> 2), y = 2 * q.y + ((a >> 1) & 1), x = 2 * q.x + (a & 1);
      s += __bfloat162float(in[((((long long)q.n * D + z) * H + y) * W + x) * C + c]);
    }
    out[i] = __float2bfloat16(0.125f * s);
  }
}
__global__ void k_pool_bwd(const float* gout, float* gin, int N, int D, int H, int W, int C, int accumulate) {
  const long long n = (long long)N * D * H * W * C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const Vox q = vox_of(i / C, D, H, W);
    const float v =
        0.125f * gout[((((long long)q.n * (D / 2) + q.z / 2) * (H / 2) + q.y / 2) * (W / 2) + q.x / 2) * C + c];
    gin[i] = accumulate ? gin[i] + v : v;
  }
}

// out = [nearest-upsample(x) (C1 channels) | skip (C2 channels)] at the fine grid, and its adjoint
__global__ void k_upcat(const bf16* x, const bf16* skip, bf16* out, int N, int D, int H, int W, int C1, int C2) {
  const int C = C1 + C2;
  const long long n = (long long)N * D * H * W * C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const long long v = i / C;
    if (c < C1) {
      const Vox q = vox_of(v, D, H, W);
      out[i] = x[((((long long)q.n * (D / 2) + q.z / 2) * (H / 2) + q.y / 2) * (W / 2) + q.x / 2) * C1 + c];
    } else {
      out[i] = skip[v * C2 + (c - C1)];
    }
  }
}
__global__ void k_upcat_bwd_x(const float* gout, float* gx, int N, int D, int H, int W, int C1, int C2) {
  // gx at the coarse grid: sum over the 8 fine children
  const int C = C1 + C2;
  const long long n = (long long)N * (D / 2) * (H / 2) * (W / 2) * C1;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C1);
    const Vox q = vox_of(i / C1, D / 2, H / 2, W / 2);
    float s = 0.0f;
    for (int a = 0; a < 8; a++) {
      const int z = 2 * q.z + (a >> 2), y = 2 * q.y + ((a >> 1) & 1), x = 2 * q.x + (a & 1);
      s += gout[((((long long)q.n * D + z) * H + y) * W + x) * C + c];
    }
    gx[i] = s;
  }
}
__global__ void k_upcat_bwd_skip(const float* gout, float* gskip, long long nvox, int C1, int C2) {
  const long long n = nvox * C2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long v = i / C2;
    gskip[i] = gout[v * (C1 + C2) + C1 + (i - v * C2)];
  }
}

// head: rho0 = sigmoid(sum_c w[c] x[c] + b); loss = mean (rho0 - target)^2 and its gradients
__global__ void k_head(const bf16* x, const float* w, const float* b, float* rho, long long nvox, int C) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox; v += (long long)gridDim.x * blockDim.x) {
    float s = b[0];
    for (int c = 0; c < C; c++) s += w[c] * __bfloat162float(x[v * C + c]);
    rho[v] = 1.0f / (1.0f + expf(-s));
  }
}
__global__ void k_head_bwd(const bf16* x, const float* w, const float* rho, const float* target, long long nvox, int C,
                           float* gx, float* part /* [gridDim.x][C + 2]: dw, db, loss */) {
  extern __shared__ float red[];  // [blockDim.x][C + 2]
  float loc[68];
  for (int c = 0; c < C + 2; c++) loc[c] = 0.0f;
  const float inv = 1.0f / (float)nvox;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox; v += (long long)gridDim.x * blockDim.x) {
    const float r = rho[v], d = r - target[v];
    const float dz = 2.0f * d * r * (1.0f - r) * inv;
    for (int c = 0; c < C; c++) {
      gx[v * C + c] = dz * w[c];
      loc[c] += dz * __bfloat162float(x[v * C + c]);
    }
    loc[C] += dz;
    loc[C + 1] += d * d * inv;
  }
  for (int c = 0; c < C + 2; c++) red[threadIdx.x * (C + 2) + c] = loc[c];
  __syncthreads();
  if (threadIdx.x < C + 2) {
    float s = 0.0f;
    for (int i = 0; i < (int)blockDim.x; i++) s += red[i * (C + 2) + threadIdx.x];
    part[blockIdx.x * (C + 2) + threadIdx.x] = s;
  }
}
__global__ void k_head_reduce(const float* part, int nblk, int n, float* out) {
  const int i = threadIdx.x;
  if (i < n) {
    float s = 0.0f;
    for (int b = 0; b < nblk; b++) s += part[b * n + i];
    out[i] = s;
  }
}

// AdamW on float32 master weights; optional bfloat16 copies in the two conv layouts
__global__ void k_adamw(float* w, const float* g, float* m, float* v, long long n, float lr, float b1, float b2,
                        float eps, float wd, float c1, float c2, bf16* wf, bf16* wb, int cin, int cout) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    float wi = w[i];
    wi -= lr * ((mi / c1) / (sqrtf(vi / c2) + eps) + wd * wi);
    w[i] = wi;
    if (wf) {  // i = (tap, ci, co)
      const long long tap = i / ((long long)cin * cout);
      const int r = (int)(i - tap * cin * cout), ci = r / cout, co = r - ci * cout;
      wf[(tap * cout + co) * cin + ci] = __float2bfloat16(wi);
      wb[(tap * cin + ci) * cout + co] = __float2bfloat16(wi);
    }
  }
}

// bfloat16 copies of float32 master conv weights [27][cin][cout]
__global__ void k_pack_w(const float* w, bf16* wf, bf16* wb, int cin, int cout) {
  const long long n = 27LL * cin * cout;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long tap = i / ((long long)cin * cout);
    const int r = (int)(i - tap * cin * cout), ci = r / cout, co = r - ci * cout;
    wf[(tap * cout + co) * cin + ci] = __float2bfloat16(w[i]);
    wb[(tap * cin + ci) * cout + co] = __float2bfloat16(w[i]);
  }
}

// network input from a target specification on the 64^3 design grid:
// channel 0 mask footprint, 1 Ht_z / Ms on the footprint, 2 plane height / 8 (all z)
__global__ void k_spec_input(const uint8_t* foot /* [N][H][W] */, const float* ht /* [N] */, const float* hgt /* [N] */,
                             bf16* out, int N, int D, int H, int W, int C) {
  const long long n = (long long)N * D * H * W;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
    const Vox q = vox_of(v, D, H, W);
    const float f = foot[((long long)q.n * H + q.y) * W + q.x] ? 1.0f : 0.0f;
    for (int c = 0; c < C; c++) {
      float val = 0.0f;
      if (c == 0) val = f;
      if (c == 1) val = f * ht[q.n];
      if (c == 2) val = hgt[q.n];
      out[v * C + c] = __float2bfloat16(val);
    }
  }
}

int grid_of(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b > 16384 ? 16384 : (b < 1 ? 1 : b));
}

int ok() { return cudaPeekAtLastError() == cudaSuccess ? 0 : -4; }

}  // namespace

extern "C" {

int tmn_conv3d_forward(const void* in, const void* Wf, const float* bias, void* out, int N, int D, int H, int W,
                       int Cin, int Cout, int relu, void* stream) {
  if (!in || !Wf || !out || Cin % 16 || (Cout != 16 && Cout != 32 && Cout != 64)) return -1;
  const long long nvox = (long long)N * D * H * W;
  const int blocks = (int)((nvox + VB - 1) / VB);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const bf16* w = reinterpret_cast<const bf16*>(Wf);
  if (Cout == 16) k_conv_mma<0, 16><<<blocks, WARPS * 32, 0, s>>>(in, w, bias, out, N, D, H, W, Cin, relu);
  if (Cout == 32) k_conv_mma<0, 32><<<blocks, WARPS * 32, 0, s>>>(in, w, bias, out, N, D, H, W, Cin, relu);
  if (Cout == 64) k_conv_mma<0, 64><<<blocks, WARPS * 32, 0, s>>>(in, w, bias, out, N, D, H, W, Cin, relu);
  return ok();
}

int tmn_conv3d_backward_data(const float* dout, const void* Wb, float* din, int N, int D, int H, int W, int Cin,
                             int Cout, int accumulate, void* stream) {
  if (!dout || !Wb || !din || Cout % 16 || (Cin != 16 && Cin != 32 && Cin != 48 && Cin != 64 && Cin != 96)) return -1;
  const long long nvox = (long long)N * D * H * W;
  const int blocks = (int)((nvox + VB - 1) / VB);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const bf16* w = reinterpret_cast<const bf16*>(Wb);
  // GEMM over k = (tap, co) with Wb[tap][ci][co]: N-side width Cin
  if (Cin == 16) k_conv_mma<1, 16><<<blocks, WARPS * 32, 0, s>>>(dout, w, nullptr, din, N, D, H, W, Cout, accumulate);
  if (Cin == 32) k_conv_mma<1, 32><<<blocks, WARPS * 32, 0, s>>>(dout, w, nullptr, din, N, D, H, W, Cout, accumulate);
  if (Cin == 48) k_conv_mma<1, 48><<<blocks, WARPS * 32, 0, s>>>(dout, w, nullptr, din, N, D, H, W, Cout, accumulate);
  if (Cin == 64) k_conv_mma<1, 64><<<blocks, WARPS * 32, 0, s>>>(dout, w, nullptr, din, N, D, H, W, Cout, accumulate);
  if (Cin == 96) k_conv_mma<1, 96><<<blocks, WARPS * 32, 0, s>>>(dout, w, nullptr, din, N, D, H, W, Cout, accumulate);
  return ok();
}

int tmn_conv3d_backward_weight(const void* in, const float* dout, float* dW, float* db, float* work,
                               long long work_floats, int N, int D, int H, int W, int Cin, int Cout, void* stream) {
  if (!in || !dout || !dW || !db || !work || Cin % 16 || Cin < 16 || (Cout != 16 && Cout != 32 && Cout != 64))
    return -1;
  const long long nvox = (long long)N * D * H * W;
  const long long chunks = (nvox + WVD - 1) / WVD;
  const long long per_blk = 27LL * Cin * Cout;
  int nblk = (int)(work_floats / per_blk);
  if (nblk > 64) nblk = 64;
  if (nblk < 1) return -5;
  const int cpb = (int)((chunks + nblk - 1) / nblk);
  nblk = (int)((chunks + cpb - 1) / cpb);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const dim3 grid(nblk, 27, Cin / 16);
  const bf16* x = reinterpret_cast<const bf16*>(in);
  if (Cout == 16) k_conv_dw_mma<2><<<grid, 128, 0, s>>>(x, dout, work, N, D, H, W, Cin, Cout, cpb);
  if (Cout == 32) k_conv_dw_mma<4><<<grid, 128, 0, s>>>(x, dout, work, N, D, H, W, Cin, Cout, cpb);
  if (Cout == 64) k_conv_dw_mma<8><<<grid, 128, 0, s>>>(x, dout, work, N, D, H, W, Cin, Cout, cpb);
  k_dw_reduce<<<grid_of(per_blk), 256, 0, s>>>(work, nblk, per_blk, dW);
  k_db<<<Cout, 256, 0, s>>>(dout, nvox, Cout, db);
  return ok();
}

int tmn_relu_backward(float* g, const void* act, long long n, void* stream) {
  k_relu_bwd<<<grid_of(n), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(g, reinterpret_cast<const bf16*>(act), n);
  return ok();
}

int tmn_pool(const void* in, void* out, int N, int D, int H, int W, int C, void* stream) {
  k_pool<<<grid_of((long long)N * D * H * W * C / 8), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      reinterpret_cast<const bf16*>(in), reinterpret_cast<bf16*>(out), N, D, H, W, C);
  return ok();
}

int tmn_pool_backward(const float* gout, float* gin, int N, int D, int H, int W, int C, int accumulate, void* stream) {
  k_pool_bwd<<<grid_of((long long)N * D * H * W * C), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      gout, gin, N, D, H, W, C, accumulate);
  return ok();
}

int tmn_upcat(const void* x, const void* skip, void* out, int N, int D, int H, int W, int C1, int C2, void* stream) {
  k_upcat<<<grid_of((long long)N * D * H * W * (C1 + C2)), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      reinterpret_cast<const bf16*>(x), reinterpret_cast<const bf16*>(skip), reinterpret_cast<bf16*>(out), N, D, H, W,
      C1, C2);
  return ok();
}

int tmn_upcat_backward(const float* gout, float* gx, float* gskip, int N, int D, int H, int W, int C1, int C2,
                       void* stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  k_upcat_bwd_x<<<grid_of((long long)N * D * H * W * C1 / 8), 256, 0, s>>>(gout, gx, N, D, H, W, C1, C2);
  k_upcat_bwd_skip<<<grid_of((long long)N * D * H * W * C2), 256, 0, s>>>(gout, gskip, (long long)N * D * H * W, C1,
                                                                        C2);
  return ok();
}

int tmn_head_forward(const void* x, const float* w, const float* b, float* rho, long long nvox, int C, void* stream) {
  k_head<<<grid_of(nvox), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(reinterpret_cast<const bf16*>(x), w, b,
                                                                             rho, nvox, C);
  return ok();
}

int tmn_head_backward(const void* x, const float* w, const float* rho, const float* target, long long nvox, int C,
                      float* gx, float* work, float* out, void* stream) {
  if (C + 2 > 68) return -1;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int nblk = 256;
  k_head_bwd<<<nblk, 128, 128 * (C + 2) * sizeof(float), s>>>(reinterpret_cast<const bf16*>(x), w, rho, target, nvox,
                                                              C, gx, work);
  k_head_reduce<<<1, 128, 0, s>>>(work, nblk, C + 2, out);
  return ok();
}

int tmn_adamw(float* w, const float* g, float* m, float* v, long long n, float lr, float b1, float b2, float eps,
              float wd, int step, void* wf, void* wb, int cin, int cout, void* stream) {
  const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
  k_adamw<<<grid_of(n), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      w, g, m, v, n, lr, b1, b2, eps, wd, c1, c2, reinterpret_cast<bf16*>(wf), reinterpret_cast<bf16*>(wb), cin, cout);
  return ok();
}

int tmn_pack_conv_weights(const float* w, void* wf, void* wb, int cin, int cout, void* stream) {
  if (!w || !wf || !wb || cin < 1 || cout < 1) return -1;
  k_pack_w<<<grid_of(27LL * cin * cout), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      w, reinterpret_cast<bf16*>(wf), reinterpret_cast<bf16*>(wb), cin, cout);
  return ok();
}

int tmn_spec_input(const uint8_t* foot, const float* ht, const float* hgt, void* out, int N, int D, int H, int W,
                   int C, void* stream) {
  k_spec_input<<<grid_of((long long)N * D * H * W), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      foot, ht, hgt, reinterpret_cast<bf16*>(out), N, D, H, W, C);
  return ok();
}

}  // extern "C"
