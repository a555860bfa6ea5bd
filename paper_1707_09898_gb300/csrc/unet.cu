// Kernels of the learned warm start: a small 3-D U-Net that maps a target
// specification to an initial density for the optimizer. Not part of the paper
// (the paper's optimizer starts from rho = 1); the optimizer always refines the
// network's output, so the network only changes how many steps are needed.
//
// Layouts: activations channels-last [N][D][H][W][C], C a multiple of 16 (padded
// channels are zero); bfloat16 activations, float32 activation gradients.
// Weights: float32 master [27][Cin][Cout] (tap = (dz+1)*9 + (dy+1)*3 + (dx+1));
// bfloat16 copies Wf (forward) and Wb (backward data) packed in the operand layout of
// the tensor-core kernels (see pack_f / pack_b below).
// 3x3x3 convolutions (stride 1, zero padding 1), forward, data gradient and weight
// gradient, are implicit GEMMs on the fifth-generation tensor cores (tcgen05.mma,
// bfloat16 operands, float32 accumulators in tensor memory): k_conv_halo (rows of 8..64
// voxels: halo rows staged once per block), k_conv_tc (any grid: per-voxel gathers) and
// k_conv_dw_tc (weight gradient, the output gradient rounded to bfloat16 as in the data
// gradient).
#include <cuda_bf16.h>
#include <stdint.h>

#include <type_traits>

#include "../../include/topomag_net.h"
#include "unet_tc.cuh"

namespace {

using bf16 = __nv_bfloat16;

__device__ __forceinline__ uint32_t pack2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
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

// Packed bfloat16 weights for the tensor-core kernels: per (tap, 16-channel chunk kc of
// the reduced dimension) a block of N x 16 values in the MMA's B layout,
// [k-group (2)][N/8][8 rows][8 elements], rows = output channels of the GEMM.
// Forward (N = cout, reduced = ci), backward data (N = cin, reduced = co).
__host__ __device__ __forceinline__ long long pack_f(int tap, int ci, int co, int cin, int cout) {
  const int kc = ci >> 4, kk = ci & 15;
  return ((long long)tap * (cin >> 4) + kc) * (16LL * cout) + (kk >> 3) * 8LL * cout + (co >> 3) * 64 + (co & 7) * 8 +
         (kk & 7);
}
__host__ __device__ __forceinline__ long long pack_b(int tap, int ci, int co, int cin, int cout) {
  const int kc = co >> 4, kk = co & 15;
  return ((long long)tap * (cout >> 4) + kc) * (16LL * cin) + (kk >> 3) * 8LL * cin + (ci >> 3) * 64 + (ci & 7) * 8 +
         (kk & 7);
}

// Error word of the tensor-core kernels: bit 0 set when a bounded wait ran out (tmn_status).
__device__ unsigned g_net_status;

// Implicit-GEMM convolution on tcgen05: a block of 128 threads owns 128 consecutive voxels
// (the M = 128 rows of the accumulator, one tensor-memory lane per voxel) and all NO output
// channels (N). The reduction runs over (tap, 16-channel chunk) steps, K = 16 each: every
// thread gathers its voxel's 16 shifted input channels into the A tile (zero outside the
// grid), thread 0 copies the step's packed weight block into the B tile (bulk copy,
// mbarrier) and issues the MMA once the step's operands are in place; S stages of A and B
// keep the next steps' loads in flight while the tensor core works. The epilogue reads
// the accumulator from tensor memory (each warp its 32 lanes).
//   MODE 0 (forward):       out[v][co] = act(sum in[v + off][ci] W[tap][ci][co] + b[co]), bfloat16
//   MODE 1 (backward data): din[v][ci] (+)= sum dout[v - off][co] W[tap][ci][co], float32
// KC: channels of the gathered input (cin forward, cout backward).
constexpr int kTcStages = 4;
template <int NO>
__host__ __device__ constexpr unsigned tmem_cols() {
  return NO <= 32 ? 32u : (NO <= 64 ? 64u : 128u);
}
template <int NO>
constexpr size_t conv_tc_smem() {
  return (size_t)kTcStages * (128 * 32 + NO * 32) + (2 * kTcStages + 1) * 8 + 16;
}
template <int MODE, int NO>
__global__ void __launch_bounds__(128) k_conv_tc(const void* src, const bf16* Wc, const float* bias, void* dst,
                                                 int Nb, int D, int H, int W, int KC, int flag) {
  using namespace tmk;
  constexpr int S = kTcStages, AB = 128 * 32, BB = NO * 32;
  constexpr unsigned NCOLS = tmem_cols<NO>();
  constexpr unsigned IDESC = idesc_bf16(128, NO);
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* As = smem;                  // [S][2 k-groups][16 row groups][8][16 B]
  unsigned char* Bs = smem + S * AB;         // [S][2][NO/8][8][16 B]
  unsigned long long* tma_bar = reinterpret_cast<unsigned long long*>(Bs + S * BB);
  unsigned long long* mma_bar = tma_bar + S;
  unsigned* tslot = reinterpret_cast<unsigned*>(mma_bar + S);
  const int t = threadIdx.x, warp = t >> 5;
  if (t == 0) {
    for (int b = 0; b < S; b++) {
      mbar_init(tma_bar + b, 1);
      mbar_init(mma_bar + b, 1);
    }
    mbar_init_fence();
  }
  if (warp == 0) {
    tmem_alloc(tslot, NCOLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned taddr = *tslot;

  const long long nvox = (long long)Nb * D * H * W;
  const long long v = (long long)blockIdx.x * 128 + t;
  const bool valid = v < nvox;
  int vx = 0, vy = 0, vz = 0, vn = 0;
  if (valid) {
    long long q = v;
    vx = (int)(q % W);
    q /= W;
    vy = (int)(q % H);
    q /= H;
    vz = (int)(q % D);
    vn = (int)(q / D);
  }
  const int nk = KC >> 4, nsteps = 27 * nk;
  // bounded waits: the first one that runs out flags g_net_status and this thread skips its
  // later waits, so a broken launch ends in milliseconds instead of spinning on every step
  bool dead = false;
  auto wait = [&](unsigned long long* mb, unsigned parity) {
    if (!dead) dead = !mbar_wait_limit(mb, parity, 1 << 16, &g_net_status);
  };
  // this thread's row (m = t) in the A tile: row group t / 8, row t % 8
  const int arow = (t >> 3) * 128 + (t & 7) * 16;
  auto load_step = [&](int s, int b) {
    const int tap = s / nk, kc = s - tap * nk;
    int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
    if (MODE == 1) {
      dz = -dz;
      dy = -dy;
      dx = -dx;
    }
    const int z = vz + dz, y = vy + dy, x = vx + dx;
    const bool ok = valid && z >= 0 && z < D && y >= 0 && y < H && x >= 0 && x < W;
    const long long u = ok ? (((long long)vn * D + z) * H + y) * W + x : 0;
    unsigned char* a = As + b * AB + arow;
    if constexpr (MODE == 0) {
      const bf16* p = reinterpret_cast<const bf16*>(src) + u * KC + kc * 16;
      cp_async16(a, p, ok ? 16u : 0u);             // channels 0..7: k-group 0
      cp_async16(a + 2048, p + 8, ok ? 16u : 0u);  // channels 8..15: k-group 1
    } else {
      uint4 lo = make_uint4(0u, 0u, 0u, 0u), hi = lo;
      if (ok) {
        const float4* p = reinterpret_cast<const float4*>(reinterpret_cast<const float*>(src) + u * KC + kc * 16);
        const float4 f0 = p[0], f1 = p[1], f2 = p[2], f3 = p[3];
        lo = make_uint4(pack2(f0.x, f0.y), pack2(f0.z, f0.w), pack2(f1.x, f1.y), pack2(f1.z, f1.w));
        hi = make_uint4(pack2(f2.x, f2.y), pack2(f2.z, f2.w), pack2(f3.x, f3.y), pack2(f3.z, f3.w));
      }
      *reinterpret_cast<uint4*>(a) = lo;
      *reinterpret_cast<uint4*>(a + 2048) = hi;
    }
    if (t == 0) {
      mbar_expect_tx(tma_bar + b, BB);
      bulk_load(Bs + b * BB, Wc + ((long long)tap * nk + kc) * NO * 16, BB, tma_bar + b);
    }
  };
  for (int s = 0; s < S - 1; s++) {  // always S - 1 groups, so that the wait below counts right
    if (s < nsteps) load_step(s, s);
    cp_async_commit();
  }
  for (int s = 0; s < nsteps; s++) {
    const int b = s % S;
    const int sn = s + S - 1;  // its loads go into the buffer the MMA of step s - 1 read
    if (sn < nsteps) {
      const int bn = sn % S;
      if (s >= 1) wait(mma_bar + bn, ((s - 1) / S) & 1);
      load_step(sn, bn);
    }
    cp_async_commit();
    cp_async_wait<S - 1>();  // this thread's copies of step s have landed
    fence_proxy_async_smem();  // its A rows, written through the generic proxy, for the tensor core
    __syncthreads();
    if (t == 0) {
      wait(tma_bar + b, (s / S) & 1);  // the weight block
      tc_fence_after();
      const uint64_t ad = smem_desc(As + b * AB, 2048, 128);
      const uint64_t bd = smem_desc(Bs + b * BB, NO * 16, 128);
      tc_mma(taddr, ad, bd, IDESC, s > 0);
      tc_commit(mma_bar + b);
    }
  }
  // the last commit arrives once every MMA has completed
  wait(mma_bar + (nsteps - 1) % S, ((nsteps - 1) / S) & 1);
  cp_async_wait<0>();
  tc_fence_after();
  const unsigned trow = taddr + ((unsigned)(warp * 32) << 16);
#pragma unroll
  for (int c0 = 0; c0 < NO; c0 += 16) {
    float r[16];
    tc_ld16(trow + c0, r);
    tc_wait_ld();
    if (!valid) continue;
    if constexpr (MODE == 0) {
      uint32_t pk[8];
#pragma unroll
      for (int i = 0; i < 8; i++) {
        float o0 = r[2 * i], o1 = r[2 * i + 1];
        if (bias) {
          o0 += bias[c0 + 2 * i];
          o1 += bias[c0 + 2 * i + 1];
        }
        if (flag) {
          o0 = fmaxf(o0, 0.0f);
          o1 = fmaxf(o1, 0.0f);
        }
        pk[i] = pack2(o0, o1);
      }
      uint4* o = reinterpret_cast<uint4*>(reinterpret_cast<bf16*>(dst) + v * NO + c0);
      o[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
      o[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
    } else {
      float4* o = reinterpret_cast<float4*>(reinterpret_cast<float*>(dst) + v * NO + c0);
#pragma unroll
      for (int i = 0; i < 4; i++) {
        float4 w = make_float4(r[4 * i], r[4 * i + 1], r[4 * i + 2], r[4 * i + 3]);
        if (flag) {  // accumulate into an existing gradient
          const float4 e = o[i];
          w.x += e.x;
          w.y += e.y;
          w.z += e.z;
          w.w += e.w;
        }
        o[i] = w;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(taddr, NCOLS);
}

template <int MODE, int NO>
int launch_conv_tc(const void* src, const bf16* Wc, const float* bias, void* dst, int Nb, int D, int H, int W, int KC,
                   int flag, cudaStream_t s) {
  constexpr size_t sm = conv_tc_smem<NO>();
  static bool init = false;
  if (!init) {
    if (cudaFuncSetAttribute(k_conv_tc<MODE, NO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
      return -4;
    init = true;
  }
  const long long nvox = (long long)Nb * D * H * W;
  const int blocks = (int)((nvox + 127) / 128);
  if (blocks > 0) k_conv_tc<MODE, NO><<<blocks, 128, sm, s>>>(src, Wc, bias, dst, Nb, D, H, W, KC, flag);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -4;
}

// Halo-tile implicit GEMM for grids whose rows hold W = 8, 16, 32 or 64 voxels (128 % W ==
// 0). A block owns TZ = 2 planes of RY = 128 / W rows of one batch item: two M = 128 tiles,
// tile m = the RY rows of plane z0 + m in (y, x) order, one tensor-memory lane per voxel.
// Per 16-channel chunk of the reduced dimension, the (TZ + 2) x (RY + 2) rows around the
// tiles are staged in shared memory once, as three copies shifted by dx = -1, 0, +1 (zero
// where x + dx leaves the grid), each in the K-major core-matrix layout
// [channel half][z][y][x][8 channels]: the A operand of tap (dz, dy, dx) for tile m is copy
// dx from row (m + dz + 1, dy + 1) on (16-byte voxel rows, row groups 128 bytes apart, the
// two channel halves one box apart), so all 27 taps read the same staged rows instead of
// gathering them again. Each staged voxel's 8 channels are read from memory once: MODE 0
// copies the unshifted rows asynchronously (all copies in flight) and builds the two
// shifted copies from them in shared memory; MODE 1 loads the float32 output gradient,
// rounds it to bfloat16 and stores it into the three copies. (TMA boxes of these 16-byte
// rows measured slower: 86 us against 77 us on a 64^3 x 2 layer.)
// The chunk's 27 packed weight blocks arrive by bulk copies (mbarrier completion). Thread 0
// issues 27 x TZ MMAs per chunk (K = 16 each); the epilogue is that of k_conv_tc. Same
// arithmetic as k_conv_tc: the same products, float32 sums in the tensor core's order.
// compile-time loop: f(std::integral_constant<int, i>) for i in [B, E)
template <int B, int E, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}
constexpr int kPartSplit = 13;  // taps [0, 13) and [13, 27) go to two accumulators
// Stage the rows (z0 - 1 + r / RP, y0 - 1 + r % RP), r < ROWS, of batch item n, channels
// [c0, c0 + 16), into three copies shifted by dx = -1, 0, +1 in the K-major core-matrix
// layout [copy][channel half][r][x][8 channels] (copy c holds x + c - 1 at position x; zero
// outside the grid), in two parts so that other loads can be in flight in between:
// stage_halo_issue copies the unshifted rows by 16-byte asynchronous copies (all in flight);
// stage_halo_finish waits for them (block barrier) and builds the shifted copies in shared
// memory. The caller still fences the generic-proxy stores for the tensor core.
template <int W, int RP, int ROWS>
__device__ __forceinline__ void stage_halo_issue(unsigned char* As, const bf16* in, int n, int z0, int y0, int D,
                                                 int H, int KC, int c0) {
  using namespace tmk;
  constexpr int BOX = 16 * W * ROWS, ITEMS = 2 * ROWS * W;
  for (int i = threadIdx.x; i < ITEMS; i += blockDim.x) {
    const int x = i % W, r = (i / W) % ROWS, h = i / (W * ROWS);
    const int z = z0 - 1 + r / RP, y = y0 - 1 + r % RP;
    const bool ok = z >= 0 && z < D && y >= 0 && y < H;
    const long long e = ok ? ((((long long)n * D + z) * H + y) * W + x) * KC + c0 + h * 8 : c0;
    cp_async16(As + (2 + h) * BOX + (r * W + x) * 16, in + e, ok ? 16u : 0u);
  }
  cp_async_commit();
}
template <int W, int ROWS>
__device__ __forceinline__ void stage_halo_finish(unsigned char* As) {
  using namespace tmk;
  constexpr int BOX = 16 * W * ROWS, ITEMS = 2 * ROWS * W;
  cp_async_wait<0>();
  __syncthreads();
  for (int i = threadIdx.x; i < ITEMS; i += blockDim.x) {
    const int x = i % W, rest = i / W, h = rest / ROWS;  // rest = h ROWS + r
    const int o = (rest - h * ROWS) * W;                 // r W
    const uint4 v = *reinterpret_cast<const uint4*>(As + (2 + h) * BOX + (o + x) * 16);
    // copy 0 at x + 1 and copy 2 at x - 1 hold this voxel; their row ends are zero
    if (x + 1 < W) *reinterpret_cast<uint4*>(As + h * BOX + (o + x + 1) * 16) = v;
    if (x >= 1) *reinterpret_cast<uint4*>(As + (4 + h) * BOX + (o + x - 1) * 16) = v;
    if (x == 0) *reinterpret_cast<uint4*>(As + h * BOX + o * 16) = make_uint4(0u, 0u, 0u, 0u);
    if (x == W - 1) *reinterpret_cast<uint4*>(As + (4 + h) * BOX + (o + W - 1) * 16) = make_uint4(0u, 0u, 0u, 0u);
  }
}

template <int W>
struct Halo {
  static constexpr int RY = 128 / W, TZ = 2, ROWS = (TZ + 2) * (RY + 2);
  static constexpr int BOX = 16 * W * ROWS;  // bytes of one channel half of one copy
  static constexpr int ABYTES = 6 * BOX;     // 3 copies x 2 halves
};
template <int NO>
__host__ __device__ constexpr int halo_cs() {  // tensor-memory columns per tile
  return NO <= 32 ? 32 : (NO <= 64 ? 64 : 128);
}
template <int W, int NO>
constexpr size_t halo_smem() {  // 128 bytes of slack to align the staged rows
  return 128 + (size_t)Halo<W>::ABYTES + 27 * NO * 32 + 2 * 8 + 16;
}
template <int MODE, int W, int NO>
__global__ void __launch_bounds__(128) k_conv_halo(const void* src, const bf16* Wc, const float* bias, void* dst,
                                                   int Nb, int D, int H, int KC, int flag) {
  using namespace tmk;
  using HT = Halo<W>;
  constexpr int RY = HT::RY, TZ = HT::TZ, ROWS = HT::ROWS, BOX = HT::BOX, BB = NO * 32, CS = halo_cs<NO>();
  constexpr unsigned NCOLS = 2 * TZ * CS;  // two accumulators (tap parts) per tile
  constexpr unsigned IDESC = idesc_bf16(128, NO);
  extern __shared__ unsigned char smem_raw[];
  unsigned char* As = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);  // [copy][half][z][y][x][16 B]
  unsigned char* Bs = As + HT::ABYTES;                                         // [tap][2][NO/8][8][16 B]
  unsigned long long* tma_bar = reinterpret_cast<unsigned long long*>(Bs + 27 * BB);
  unsigned long long* mma_bar = tma_bar + 1;
  unsigned* tslot = reinterpret_cast<unsigned*>(mma_bar + 1);
  const int t = threadIdx.x, warp = t >> 5;
  const int nyt = (H + RY - 1) / RY, nzt = (D + TZ - 1) / TZ;
  const int yt = blockIdx.x % nyt, zt = (blockIdx.x / nyt) % nzt, n = blockIdx.x / (nyt * nzt);
  const int y0 = yt * RY, z0 = zt * TZ;
  if (t == 0) {
    mbar_init(tma_bar, 1);
    mbar_init(mma_bar, 2 * TZ);  // one commit per issuer
    mbar_init_fence();
  }
  if (warp == 0) {
    tmem_alloc(tslot, NCOLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned taddr = *tslot;
  bool dead = false;
  auto wait = [&](unsigned long long* mb, unsigned parity) {
    if (!dead) dead = !mbar_wait_limit(mb, parity, 1 << 16, &g_net_status);
  };
  const int nk = KC >> 4;
  for (int kc = 0; kc < nk; kc++) {
    if (kc > 0) wait(mma_bar, (kc - 1) & 1);  // the MMAs of the previous chunk have read the buffers
    if (t == 0) {
      if (kc == 0) fence_proxy_async_global();  // the source was written by ordinary stores
      fence_proxy_async_smem();
      mbar_expect_tx(tma_bar, 27 * BB);
      for (int tap = 0; tap < 27; tap++) bulk_load(Bs + tap * BB, Wc + ((long long)tap * nk + kc) * NO * 16, BB, tma_bar);
    }
    if constexpr (MODE == 0) {
      stage_halo_issue<W, RY + 2, ROWS>(As, reinterpret_cast<const bf16*>(src), n, z0, y0, D, H, KC, kc * 16);
      stage_halo_finish<W, ROWS>(As);
    } else {
      // (half, row, x) items, x fastest: the 8 float32 values of one voxel are read once,
      // rounded to bfloat16 and stored into the copies that hold them (copy c has the value
      // of x + c - 1 at position x); the loads of kBatch items are in flight together
      constexpr int XW = W + 2, ITEMS = 2 * ROWS * XW, kBatch = 8;
      constexpr int NV = MODE == 0 ? 1 : 2;  // 16-byte loads per item (MODE 1: 8 float32 values)
      for (int i0 = 0; i0 < ITEMS; i0 += 128 * kBatch) {
        uint4 raw[kBatch][NV];  // loaded first, converted after the batch's loads are issued
#pragma unroll
        for (int b = 0; b < kBatch; b++) {
          const int i = i0 + b * 128 + t;
          const int x = i % XW - 1, r = (i / XW) % ROWS, h = i / (XW * ROWS);
          const int z = z0 - 1 + r / (RY + 2), y = y0 - 1 + r % (RY + 2);
#pragma unroll
          for (int v = 0; v < NV; v++) raw[b][v] = make_uint4(0u, 0u, 0u, 0u);
          if (i < ITEMS && z >= 0 && z < D && y >= 0 && y < H && x >= 0 && x < W) {
            const long long e = ((((long long)n * D + z) * H + y) * W + x) * KC + kc * 16 + h * 8;
            const uint4* q = MODE == 0 ? reinterpret_cast<const uint4*>(reinterpret_cast<const bf16*>(src) + e)
                                       : reinterpret_cast<const uint4*>(reinterpret_cast<const float*>(src) + e);
#pragma unroll
            for (int v = 0; v < NV; v++) raw[b][v] = q[v];
          }
        }
#pragma unroll
        for (int b = 0; b < kBatch; b++) {
          const int i = i0 + b * 128 + t;
          const int x = i % XW - 1, r = (i / XW) % ROWS, h = i / (XW * ROWS);
          uint4 pk = raw[b][0];
          if constexpr (MODE == 1) {
            const float4 f0 = *reinterpret_cast<const float4*>(&raw[b][0]);
            const float4 f1 = *reinterpret_cast<const float4*>(&raw[b][NV - 1]);
            pk = make_uint4(pack2(f0.x, f0.y), pack2(f0.z, f0.w), pack2(f1.x, f1.y), pack2(f1.z, f1.w));
          }
#pragma unroll
          for (int c = 0; c < 3; c++) {
            const int xs = x + 1 - c;
            if (i < ITEMS && xs >= 0 && xs < W)
              *reinterpret_cast<uint4*>(As + (c * 2 + h) * BOX + (r * W + xs) * 16) = pk;
          }
        }
      }
    }
    fence_proxy_async_smem();  // the staged rows, written through the generic proxy, for the tensor core
    __syncthreads();
    if ((t & 31) == 0) {
      // lane 0 of warp w issues the MMAs of tile m = w % TZ for the taps of part w / TZ into
      // that part's own accumulator (the issue of one MMA takes tens of cycles, so four
      // issuers work side by side; the epilogue adds the parts); descriptors are a base plus
      // compile-time offsets (16-byte units; every address stays below 2^18 bytes)
      const int m = warp % TZ, part = warp / TZ;
      wait(tma_bar, kc & 1);
      tc_fence_after();
      const uint64_t a0 = smem_desc(As + m * (RY + 2) * W * 16, BOX, 128);
      const uint64_t b0 = smem_desc(Bs, NO * 16, 128);
      const unsigned acc = taddr + (part * TZ + m) * CS;
      auto issue = [&](auto tap_c) {
        constexpr int tap = decltype(tap_c)::value;
        constexpr int sg = MODE == 1 ? -1 : 1;
        constexpr int dz = sg * (tap / 9 - 1), dy = sg * ((tap / 3) % 3 - 1), dx = sg * (tap % 3 - 1);
        constexpr unsigned aoff = (unsigned)((dx + 1) * 2 * BOX + ((dz + 1) * (RY + 2) + dy + 1) * W * 16) >> 4;
        tc_mma(acc, a0 + aoff, b0 + (unsigned)(tap * BB >> 4), IDESC, kc > 0 || (tap != 0 && tap != kPartSplit));
      };
      if (part == 0) {
        static_for<0, kPartSplit>(issue);
      } else {
        static_for<kPartSplit, 27>(issue);
      }
      tc_commit(mma_bar);
    }
  }
  wait(mma_bar, (nk - 1) & 1);  // every MMA has completed
  tc_fence_after();
  const unsigned trow = taddr + ((unsigned)(warp * 32) << 16);
  const int y = y0 + t / W, x = t % W;
#pragma unroll
  for (int m = 0; m < TZ; m++) {
    const int z = z0 + m;
    const bool valid = z < D && y < H;
    const long long v = (((long long)n * D + z) * H + y) * W + x;
#pragma unroll
    for (int c0 = 0; c0 < NO; c0 += 16) {
      float r[16], r2[16];
      tc_ld16(trow + m * CS + c0, r);
      tc_ld16(trow + (TZ + m) * CS + c0, r2);
      tc_wait_ld();
      if (!valid) continue;
#pragma unroll
      for (int i = 0; i < 16; i++) r[i] += r2[i];  // taps 0 .. 12 and 13 .. 26
      if constexpr (MODE == 0) {
        uint32_t pk[8];
#pragma unroll
        for (int i = 0; i < 8; i++) {
          float o0 = r[2 * i], o1 = r[2 * i + 1];
          if (bias) {
            o0 += bias[c0 + 2 * i];
            o1 += bias[c0 + 2 * i + 1];
          }
          if (flag) {
            o0 = fmaxf(o0, 0.0f);
            o1 = fmaxf(o1, 0.0f);
          }
          pk[i] = pack2(o0, o1);
        }
        uint4* o = reinterpret_cast<uint4*>(reinterpret_cast<bf16*>(dst) + v * NO + c0);
        o[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        o[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
      } else {
        float4* o = reinterpret_cast<float4*>(reinterpret_cast<float*>(dst) + v * NO + c0);
#pragma unroll
        for (int i = 0; i < 4; i++) {
          float4 w = make_float4(r[4 * i], r[4 * i + 1], r[4 * i + 2], r[4 * i + 3]);
          if (flag) {  // accumulate into an existing gradient
            const float4 e = o[i];
            w.x += e.x;
            w.y += e.y;
            w.z += e.z;
            w.w += e.w;
          }
          o[i] = w;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(taddr, NCOLS);
}

template <int MODE, int W, int NO>
int launch_conv_halo(const void* src, const bf16* Wc, const float* bias, void* dst, int Nb, int D, int H, int KC,
                     int flag, cudaStream_t s) {
  using HT = Halo<W>;
  constexpr size_t sm = halo_smem<W, NO>();
  static_assert(sm <= 227 * 1024, "shared memory of one block");
  static bool init = false;
  if (!init) {
    if (cudaFuncSetAttribute(k_conv_halo<MODE, W, NO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) !=
        cudaSuccess)
      return -4;
    init = true;
  }
  const long long blocks = (long long)Nb * ((D + HT::TZ - 1) / HT::TZ) * ((H + HT::RY - 1) / HT::RY);
  if (blocks > 0x7fffffffLL) return -1;
  if (blocks > 0)
    k_conv_halo<MODE, W, NO><<<(unsigned)blocks, 128, sm, s>>>(src, Wc, bias, dst, Nb, D, H, KC, flag);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -4;
}

// the halo kernel for rows of 8 .. 64 voxels, else the per-voxel gather kernel
template <int MODE, int NO>
int launch_conv(const void* src, const bf16* Wc, const float* bias, void* dst, int Nb, int D, int H, int W, int KC,
                int flag, cudaStream_t s) {
  if ((reinterpret_cast<uintptr_t>(src) & 15) == 0) {
    if (W == 64) return launch_conv_halo<MODE, 64, NO>(src, Wc, bias, dst, Nb, D, H, KC, flag, s);
    if (W == 32) return launch_conv_halo<MODE, 32, NO>(src, Wc, bias, dst, Nb, D, H, KC, flag, s);
    if (W == 16) return launch_conv_halo<MODE, 16, NO>(src, Wc, bias, dst, Nb, D, H, KC, flag, s);
    if (W == 8) return launch_conv_halo<MODE, 8, NO>(src, Wc, bias, dst, Nb, D, H, KC, flag, s);
  }
  return launch_conv_tc<MODE, NO>(src, Wc, bias, dst, Nb, D, H, W, KC, flag, s);
}

// Weight gradient on tcgen05: dW[tap][ci][co] = sum_v in[v + off(tap)][ci] q(dout[v][co]),
// a GEMM with rows (tap, ci), columns co and the voxels as the reduction. A block owns one
// row tile of 128 = 8 taps x 16 input channels (tile = (tap group, channel chunk)) and a
// range of voxels, 16 per MMA (K = 16), kDwChunks MMAs per pipeline stage; its float32
// accumulator (128 x NO) lives in tensor memory and is written out as one partial, and
// k_dw_reduce_tc adds the partials in block order. Both operands are MN-major, so the channels-last rows go into shared memory as
// they are: A gets each (tap, voxel)'s 16 shifted input channels (two 16-byte pieces), B
// each voxel's NO output-gradient channels, taken from a bfloat16 copy made beforehand
// (rounded to nearest even, the operand precision of every product).
constexpr int kDwStages = 3, kDwChunks = 4;  // pipeline stages; 16-voxel chunks (MMAs) per stage
constexpr int kDwBlocksPerSm = 4;            // voxel blocks per SM, over all row tiles
template <int NO>
constexpr size_t dw_tc_smem() {
  return (size_t)kDwStages * kDwChunks * (128 * 32 + NO * 32) + (2 * kDwStages + 1) * 8 + 16;
}
template <int NO>
__global__ void __launch_bounds__(128) k_conv_dw_tc(const bf16* in, const bf16* g16, float* part, int Nb, int D,
                                                    int H, int W, int Cin, long long chunks_per_block) {
  using namespace tmk;
  constexpr int S = kDwStages, KS = kDwChunks, AB = 128 * 32, BB = NO * 32, PG = NO / 8;
  constexpr unsigned NCOLS = tmem_cols<NO>();
  constexpr unsigned IDESC = idesc_bf16(128, NO, true);
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* As = smem;                // [S][KS][k-group (2)][16 row groups][8 k-rows][16 B]
  unsigned char* Bs = smem + S * KS * AB;  // [S][KS][2][PG][8][16 B]
  unsigned long long* mma_bar = reinterpret_cast<unsigned long long*>(Bs + S * KS * BB);
  unsigned* tslot = reinterpret_cast<unsigned*>(mma_bar + S);
  const int t = threadIdx.x, warp = t >> 5;
  if (t == 0) {
    for (int b = 0; b < S; b++) mbar_init(mma_bar + b, 1);
    mbar_init_fence();
  }
  if (warp == 0) {
    tmem_alloc(tslot, NCOLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned taddr = *tslot;
  bool dead = false;
  auto wait = [&](unsigned long long* mb, unsigned parity) {
    if (!dead) dead = !mbar_wait_limit(mb, parity, 1 << 16, &g_net_status);
  };
  const long long nvox = (long long)Nb * D * H * W;
  const int tile = blockIdx.y, ncc = Cin >> 4;
  const int tg = tile / ncc, cc = tile - tg * ncc;
  // A: this thread's (tap, voxel) = (8 tg + t / 16, t % 16) of each chunk
  const int tap = 8 * tg + (t >> 4), ka = t & 15;
  const bool tap_ok = tap < 27;
  const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
  const int aoff = (t >> 4) * 2 * 128 + (ka >> 3) * 2048 + (ka & 7) * 16;
  // B: this thread's piece (voxel kb, 8 channels pg) of each chunk, if t < 16 PG
  const int kb = t / PG, pg = t - kb * PG;
  const int boff = pg * 128 + (kb >> 3) * (PG * 128) + (kb & 7) * 16;
  const long long c0 = (long long)blockIdx.x * chunks_per_block;
  const long long nch = (nvox + 15) / 16;
  const long long c1 = c0 + chunks_per_block < nch ? c0 + chunks_per_block : nch;
  const int nsteps = c1 > c0 ? (int)((c1 - c0 + KS - 1) / KS) : 0;
  // this thread's A voxel v = 16 ch + ka as a cursor (x, y, z, n) that the steps advance by
  // 16 voxels in order (no divisions in the loop)
  int cx = 0, cy = 0, cz = 0;
  long long cn = 0;
  {
    long long q = c0 * 16 + ka;
    cx = (int)(q % W);
    q /= W;
    cy = (int)(q % H);
    q /= H;
    cz = (int)(q % D);
    cn = q / D;
  }
  // step s: chunks c0 + s KS + k (k < KS) of the block's range; chunks past it read zeros
  auto load_step = [&](int s, int b) {
#pragma unroll
    for (int k = 0; k < KS; k++) {
      const long long ch = c0 + (long long)s * KS + k;
      const long long v0 = ch * 16;
      const bool in_range = ch < c1;
      {
        const long long v = v0 + ka;
        const int x = cx + dx, y = cy + dy, z = cz + dz;
        const bool ok = in_range && tap_ok && v < nvox && z >= 0 && z < D && y >= 0 && y < H && x >= 0 && x < W;
        const long long u = ok ? ((cn * D + z) * H + y) * W + x : 0;
        cx += 16;  // the cursor moves to this thread's voxel of the next chunk
        while (cx >= W) {
          cx -= W;
          if (++cy == H) {
            cy = 0;
            if (++cz == D) {
              cz = 0;
              ++cn;
            }
          }
        }
        const bf16* src = in + u * Cin + cc * 16;
        unsigned char* a = As + (b * KS + k) * AB + aoff;
        cp_async16(a, src, ok ? 16u : 0u);            // channels 0..7: row group 2 (t / 16)
        cp_async16(a + 128, src + 8, ok ? 16u : 0u);  // channels 8..15: the next row group
      }
      if (t < 16 * PG) {
        const long long v = v0 + kb;
        const bool ok = in_range && v < nvox;
        cp_async16(Bs + (b * KS + k) * BB + boff, g16 + (ok ? v : 0) * NO + pg * 8, ok ? 16u : 0u);
      }
    }
  };
  for (int s = 0; s < S - 1; s++) {  // always S - 1 groups, so that the wait below counts right
    if (s < nsteps) load_step(s, s);
    cp_async_commit();
  }
  for (int s = 0; s < nsteps; s++) {
    const int b = s % S;
    const int sn = s + S - 1;
    if (sn < nsteps) {
      const int bn = sn % S;
      if (s >= 1) wait(mma_bar + bn, ((s - 1) / S) & 1);
      load_step(sn, bn);
    }
    cp_async_commit();
    cp_async_wait<S - 1>();
    fence_proxy_async_smem();
    __syncthreads();
    if (t == 0) {
      tc_fence_after();
#pragma unroll
      for (int k = 0; k < KS; k++) {
        const uint64_t ad = smem_desc(As + (b * KS + k) * AB, 2048, 128);
        const uint64_t bd = smem_desc(Bs + (b * KS + k) * BB, PG * 128, 128);
        tc_mma(taddr, ad, bd, IDESC, s > 0 || k > 0);
      }
      tc_commit(mma_bar + b);
    }
  }
  if (nsteps > 0) wait(mma_bar + (nsteps - 1) % S, ((nsteps - 1) / S) & 1);
  cp_async_wait<0>();
  tc_fence_after();
  // row t of the tile: tap 8 tg + t / 16, channel 16 cc + t % 16
  float* pr = part + (((long long)blockIdx.x * gridDim.y + tile) * 128 + t) * NO;
  const unsigned trow = taddr + ((unsigned)(warp * 32) << 16);
#pragma unroll
  for (int q0 = 0; q0 < NO; q0 += 16) {
    float r[16];
    tc_ld16(trow + q0, r);
    tc_wait_ld();
#pragma unroll
    for (int i = 0; i < 16; i++) r[i] = nsteps > 0 ? r[i] : 0.0f;
    float4* o = reinterpret_cast<float4*>(pr + q0);
#pragma unroll
    for (int i = 0; i < 4; i++) o[i] = make_float4(r[4 * i], r[4 * i + 1], r[4 * i + 2], r[4 * i + 3]);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(taddr, NCOLS);
}

// Weight gradient for rows of 8..64 voxels (128 % W == 0): dW[tap][ci][co] =
// sum_v in[v + off(tap)][ci] q(dout[v][co]) as MMAs with M = co (padded to 128), N = the
// 16 input channels of a chunk for the three dx taps at once (48), K = 16 voxels. A
// persistent block takes tiles of one plane x 128 / W rows (128 voxels): it stages the three
// planes of rows around the tile once, in the forward's three dx-shifted copies, whose
// channel halves and dx copies lie one box apart -- the uniform stride the N side needs --
// and the tile's output gradient, rounded to bfloat16, as [8 co][voxel] rows. Each of the
// nine (dz, dy) pairs then has one accumulator of 48 tensor-memory columns (432 in all),
// fed by 8 MMAs per tile from four issuing threads. After the block's tiles of a channel
// chunk its accumulators go out as one float32 partial per block; k_dw_reduce_halo adds the
// partials in block order. Same products as k_conv_dw_tc, float32 sums in another order.
template <int W>
struct DwHalo {
  static constexpr int RY = 128 / W, NV = 128, ROWS = 3 * (RY + 2);
  static constexpr int BOX = 16 * W * ROWS, ABYTES = 6 * BOX, GBYTES = 16 * NV * 16;
};
template <int W>
constexpr size_t dw_halo_smem() {
  return 128 + (size_t)DwHalo<W>::ABYTES + DwHalo<W>::GBYTES + 2 * 8 + 16;
}
template <int W, int NO>
__global__ void __launch_bounds__(128, 1) k_conv_dw_halo(const bf16* in, const float* dout, float* part, int Nb,
                                                         int D, int H, int Cin) {
  using namespace tmk;
  using HT = DwHalo<W>;
  constexpr int RY = HT::RY, NV = HT::NV, ROWS = HT::ROWS, BOX = HT::BOX;
  constexpr unsigned NCOLS = 512, IDESC = idesc_bf16(128, 48, true);
  extern __shared__ unsigned char smem_raw[];
  unsigned char* As = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);  // [copy][half][plane][y][x][16 B]
  unsigned char* Gs = As + HT::ABYTES;                                         // [16 co groups][NV][16 B]
  unsigned long long* mma_bar = reinterpret_cast<unsigned long long*>(Gs + HT::GBYTES);
  unsigned* tslot = reinterpret_cast<unsigned*>(mma_bar + 1);
  const int t = threadIdx.x, warp = t >> 5;
  for (int i = t; i < (16 - NO / 8) * NV; i += 128)  // co >= NO: zero rows of A, never written again
    *reinterpret_cast<uint4*>(Gs + (NO / 8) * NV * 16 + i * 16) = make_uint4(0u, 0u, 0u, 0u);
  if (t == 0) {
    mbar_init(mma_bar, 4);  // one commit per issuer
    mbar_init_fence();
  }
  if (warp == 0) {
    tmem_alloc(tslot, NCOLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned taddr = *tslot;
  bool dead = false;
  auto wait = [&](unsigned long long* mb, unsigned parity) {
    if (!dead) dead = !mbar_wait_limit(mb, parity, 1 << 16, &g_net_status);
  };
  const int nyt = (H + RY - 1) / RY;
  const long long ntiles = (long long)Nb * D * nyt;
  const int nk = Cin >> 4;
  unsigned phase = 0;  // completed phases of mma_bar
  for (int kc = 0; kc < nk; kc++) {
    bool first = true;  // the block's first tile of this chunk starts the accumulators
    for (long long q = blockIdx.x; q < ntiles; q += gridDim.x) {
      const int yt = (int)(q % nyt);
      const long long rq = q / nyt;
      const int z = (int)(rq % D), n = (int)(rq / D), y0 = yt * RY;
      if (!first) {  // the previous tile's MMAs have read the staged rows
        wait(mma_bar, phase & 1);
        phase++;
      }
      if (t == 0 && kc == 0 && first) fence_proxy_async_global();  // in and dout came by ordinary stores
      stage_halo_issue<W, RY + 2, ROWS>(As, in, n, z, y0, D, H, Cin, kc * 16);  // in flight meanwhile
      // the tile's output gradient: voxel v = ty W + x, co group cg; zero outside the grid
      {
        constexpr int GI = NV * (NO / 8);
        for (int i = t; i < GI; i += 128) {
          const int v = i % NV, cg = i / NV, y = y0 + v / W;
          uint4 pk = make_uint4(0u, 0u, 0u, 0u);
          if (y < H) {
            const float4* g = reinterpret_cast<const float4*>(
                dout + ((((long long)n * D + z) * H + y) * W + v % W) * NO + cg * 8);
            const float4 f0 = g[0], f1 = g[1];
            pk = make_uint4(pack2(f0.x, f0.y), pack2(f0.z, f0.w), pack2(f1.x, f1.y), pack2(f1.z, f1.w));
          }
          *reinterpret_cast<uint4*>(Gs + cg * NV * 16 + v * 16) = pk;
        }
      }
      stage_halo_finish<W, ROWS>(As);
      fence_proxy_async_smem();  // the staged rows, written through the generic proxy, for the tensor core
      __syncthreads();
      if ((t & 31) == 0) {
        // issuer w: the (dz, dy) pairs w, w + 4, w + 8 (nine over four issuers)
        tc_fence_after();
        const uint64_t a0 = smem_desc(Gs, 128, NV * 16);  // K groups (8 voxels) 128 B, M groups (8 co) NV 16 B
        const uint64_t b0 = smem_desc(As, 128, BOX);      // K groups 128 B, N groups (half, then dx) one box
        for (int p = warp; p < 9; p += 4) {
          const int dz = p / 3 - 1, dy = p % 3 - 1;
#pragma unroll
          for (int ks = 0; ks < NV / 16; ks++) {
            const int v0 = ks * 16, ty = v0 / W, x0 = v0 % W;
            const unsigned boff = (unsigned)((((dz + 1) * (RY + 2) + ty + dy + 1) * W + x0) * 16) >> 4;
            tc_mma(taddr + p * 48, a0 + (unsigned)(v0 * 16 >> 4), b0 + boff, IDESC, !(first && ks == 0));
          }
        }
        tc_commit(mma_bar);
      }
      first = false;
    }
    if (!first) {
      wait(mma_bar, phase & 1);
      phase++;
    }
    tc_fence_after();
    // the chunk's partial: lane co of warp co / 32 holds D[co][dx 16 + ci] of pair p
    float* pb = part + (long long)blockIdx.x * 27 * Cin * NO;
    if (warp * 32 < NO) {
      const int co = t;
#pragma unroll 1
      for (int p = 0; p < 9; p++) {
#pragma unroll
        for (int dxi = 0; dxi < 3; dxi++) {
          float r[16];
          tc_ld16(taddr + ((unsigned)(warp * 32) << 16) + p * 48 + dxi * 16, r);
          tc_wait_ld();
          const int tap = p * 3 + dxi;  // (dz + 1) 9 + (dy + 1) 3 + (dx + 1)
          if (co < NO) {
#pragma unroll
            for (int i = 0; i < 16; i++) pb[((long long)tap * Cin + kc * 16 + i) * NO + co] = first ? 0.0f : r[i];
          }
        }
      }
    }
    tc_fence_before();
    __syncthreads();  // the accumulators are read before the next chunk's MMAs overwrite them
    tc_fence_after();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(taddr, NCOLS);
}

// dW = sum over the blocks p (in order) of part[p][tap][ci][co]
__global__ void k_dw_reduce_halo(const float* part, int nblk, long long n, float* dW) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int b = 0; b < nblk; b++) s += part[(long long)b * n + i];
    dW[i] = s;
  }
}

// dW[tap][ci][co] = sum over the voxel blocks p (in order) of part[p][tile][row][co]
__global__ void k_dw_reduce_tc(const float* part, int nblk, int ntiles, int Cin, int Cout, float* dW) {
  const long long n = 27LL * Cin * Cout;
  const int ncc = Cin >> 4;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int tap = (int)(i / ((long long)Cin * Cout));
    const int r = (int)(i - (long long)tap * Cin * Cout), ci = r / Cout, co = r - ci * Cout;
    const int tile = (tap >> 3) * ncc + (ci >> 4), row = (tap & 7) * 16 + (ci & 15);
    float s = 0.0f;
    for (int b = 0; b < nblk; b++) s += part[(((long long)b * ntiles + tile) * 128 + row) * Cout + co];
    dW[i] = s;
  }
}

// bfloat16 copy of a float32 array (round to nearest even), two values per thread step
__global__ void k_to_bf16(const float* x, bf16* y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; 2 * i < n; i += (long long)gridDim.x * blockDim.x) {
    if (2 * i + 1 < n) {
      *reinterpret_cast<uint32_t*>(y + 2 * i) = pack2(x[2 * i], x[2 * i + 1]);
    } else {
      y[2 * i] = __float2bfloat16(x[2 * i]);
    }
  }
}

// the bias gradient: float32 sum over the voxels of the unrounded output gradient
// The bias gradient db[c] = sum over the voxels of dout[v][c] (float32, unrounded), in a
// fixed order: block b sums its range of voxels for every channel (consecutive threads on
// consecutive channels, then voxels), k_db_final adds the block partials in block order.
constexpr int kDbBlocks = 256;
__global__ void __launch_bounds__(256) k_db_part(const float* dout, long long nvox, int C, float* part) {
  __shared__ float red[256];
  const int t = threadIdx.x, c = t % C, lane = t / C, lanes = 256 / C;
  const long long chunk = (nvox + gridDim.x - 1) / gridDim.x;
  const long long v0 = blockIdx.x * chunk, v1 = v0 + chunk < nvox ? v0 + chunk : nvox;
  float s = 0.0f;
  for (long long v = v0 + lane; v < v1; v += lanes) s += dout[v * C + c];
  red[t] = s;
  __syncthreads();
  if (t < C) {
    float a = 0.0f;
    for (int l = 0; l < lanes; l++) a += red[l * C + t];
    part[(long long)blockIdx.x * C + t] = a;
  }
}
__global__ void k_db_final(const float* part, int nblk, int C, float* db) {
  if ((int)threadIdx.x < C) {
    float a = 0.0f;
    for (int b = 0; b < nblk; b++) a += part[(long long)b * C + threadIdx.x];
    db[threadIdx.x] = a;
  }
}
// after the weight gradient's partials are consumed, work holds the bias partials
int launch_db(const float* dout, long long nvox, int C, float* work, float* db, cudaStream_t s) {
  const int nb = (int)(nvox < kDbBlocks ? nvox : kDbBlocks);
  k_db_part<<<nb, 256, 0, s>>>(dout, nvox, C, work);
  k_db_final<<<1, 64, 0, s>>>(work, nb, C, db);
  return 0;
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
      const int tap = (int)(i / ((long long)cin * cout));
      const int r = (int)(i - (long long)tap * cin * cout), ci = r / cout, co = r - ci * cout;
      wf[pack_f(tap, ci, co, cin, cout)] = __float2bfloat16(wi);
      wb[pack_b(tap, ci, co, cin, cout)] = __float2bfloat16(wi);
    }
  }
}

// bfloat16 copies of float32 master conv weights [27][cin][cout]
__global__ void k_pack_w(const float* w, bf16* wf, bf16* wb, int cin, int cout) {
  const long long n = 27LL * cin * cout;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int tap = (int)(i / ((long long)cin * cout));
    const int r = (int)(i - (long long)tap * cin * cout), ci = r / cout, co = r - ci * cout;
    wf[pack_f(tap, ci, co, cin, cout)] = __float2bfloat16(w[i]);
    wb[pack_b(tap, ci, co, cin, cout)] = __float2bfloat16(w[i]);
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
  if (!in || !Wf || !out || Cin % 16 || Cin < 16 || (Cout != 16 && Cout != 32 && Cout != 64)) return -1;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const bf16* w = reinterpret_cast<const bf16*>(Wf);
  if (Cout == 16) return launch_conv<0, 16>(in, w, bias, out, N, D, H, W, Cin, relu, s);
  if (Cout == 32) return launch_conv<0, 32>(in, w, bias, out, N, D, H, W, Cin, relu, s);
  return launch_conv<0, 64>(in, w, bias, out, N, D, H, W, Cin, relu, s);
}

int tmn_conv3d_backward_data(const float* dout, const void* Wb, float* din, int N, int D, int H, int W, int Cin,
                             int Cout, int accumulate, void* stream) {
  if (!dout || !Wb || !din || Cout % 16 || Cout < 16 || (Cin != 16 && Cin != 32 && Cin != 48 && Cin != 64 && Cin != 96))
    return -1;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const bf16* w = reinterpret_cast<const bf16*>(Wb);
  // GEMM over k = (tap, co) with the output channels ci as the N side
  if (Cin == 16) return launch_conv<1, 16>(dout, w, nullptr, din, N, D, H, W, Cout, accumulate, s);
  if (Cin == 32) return launch_conv<1, 32>(dout, w, nullptr, din, N, D, H, W, Cout, accumulate, s);
  if (Cin == 48) return launch_conv<1, 48>(dout, w, nullptr, din, N, D, H, W, Cout, accumulate, s);
  if (Cin == 64) return launch_conv<1, 64>(dout, w, nullptr, din, N, D, H, W, Cout, accumulate, s);
  return launch_conv<1, 96>(dout, w, nullptr, din, N, D, H, W, Cout, accumulate, s);
}

int tmn_status(unsigned* out) {
  if (!out) return -1;
  unsigned z = 0;
  if (cudaMemcpyFromSymbol(out, g_net_status, sizeof(unsigned)) != cudaSuccess) return -4;
  if (cudaMemcpyToSymbol(g_net_status, &z, sizeof(unsigned)) != cudaSuccess) return -4;
  return 0;
}

long long tmn_conv3d_backward_weight_work(long long nvox, int Cin, int Cout) {
  if (nvox < 1 || Cin < 16 || Cin % 16 || Cout < 16 || Cout % 16) return -1;
  const long long copy = (nvox * Cout + 1) / 2;         // floats holding the bfloat16 copy of dout
  return (copy + 3) / 4 * 4 + 4LL * (Cin / 16) * 128 * Cout;  // partials from a 16-byte boundary, one set
}

int tmn_conv3d_backward_weight(const void* in, const float* dout, float* dW, float* db, float* work,
                               long long work_floats, int N, int D, int H, int W, int Cin, int Cout, void* stream) {
  if (!in || !dout || !dW || !db || !work || Cin % 16 || Cin < 16 || (Cout != 16 && Cout != 32 && Cout != 64))
    return -1;
  const long long nvox = (long long)N * D * H * W;
  if (nvox < 1) return -1;
  if (work_floats < tmn_conv3d_backward_weight_work(nvox, Cin, Cout)) return -5;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) nsm = 148;
  }
  if ((W == 8 || W == 16 || W == 32 || W == 64) && (reinterpret_cast<uintptr_t>(in) & 15) == 0) {
    // halo tiles: one persistent block per SM, as many as the work buffer holds partials for
    const long long per = 27LL * Cin * Cout, ntl = (long long)N * D * ((H + 128 / W - 1) / (128 / W));
    long long nblk = work_floats / per;
    if (nblk > nsm) nblk = nsm;
    if (nblk > ntl) nblk = ntl;
    const bf16* x = reinterpret_cast<const bf16*>(in);
    int r = 0;
    auto run = [&](auto kernel, size_t sm) {
      if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
        r = -4;
      else
        kernel<<<(unsigned)nblk, 128, sm, s>>>(x, dout, work, N, D, H, Cin);
    };
#define TMN_DW_HALO(WW)                                                             \
  if (W == WW) {                                                                    \
    if (Cout == 16) run(k_conv_dw_halo<WW, 16>, dw_halo_smem<WW>());                \
    if (Cout == 32) run(k_conv_dw_halo<WW, 32>, dw_halo_smem<WW>());                \
    if (Cout == 64) run(k_conv_dw_halo<WW, 64>, dw_halo_smem<WW>());                \
  }
    TMN_DW_HALO(8)
    TMN_DW_HALO(16)
    TMN_DW_HALO(32)
    TMN_DW_HALO(64)
#undef TMN_DW_HALO
    if (r) return r;
    k_dw_reduce_halo<<<grid_of(per), 256, 0, s>>>(work, (int)nblk, per, dW);
    launch_db(dout, nvox, Cout, work, db, s);
    return ok();
  }
  const long long pofs = ((nvox * Cout + 1) / 2 + 3) / 4 * 4;
  const int tiles = 4 * (Cin / 16);
  const long long per_blk = (long long)tiles * 128 * Cout;
  // voxel blocks: about four blocks per SM over all tiles (each block's loop is bound by the
  // latency of its gathers, so several of them in flight), no more than the work buffer holds
  const long long chunks = (nvox + 15) / 16;
  long long nblk = (work_floats - pofs) / per_blk;
  const long long want = ((long long)kDwBlocksPerSm * nsm + tiles - 1) / tiles;
  if (nblk > want) nblk = want;
  if (nblk > chunks) nblk = chunks;
  long long cpb = (chunks + nblk - 1) / nblk;
  if (cpb > kDwChunks) cpb = (cpb + kDwChunks - 1) / kDwChunks * kDwChunks;  // whole pipeline stages
  nblk = (chunks + cpb - 1) / cpb;
  bf16* g16 = reinterpret_cast<bf16*>(work);
  float* part = work + pofs;
  k_to_bf16<<<grid_of(nvox * Cout / 2 + 1), 256, 0, s>>>(dout, g16, nvox * Cout);
  const dim3 grid((unsigned)nblk, (unsigned)tiles);
  const bf16* x = reinterpret_cast<const bf16*>(in);
  int r = 0;
  auto run = [&](auto kernel, size_t sm) {
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
      r = -4;
    else
      kernel<<<grid, 128, sm, s>>>(x, g16, part, N, D, H, W, Cin, cpb);
  };
  if (Cout == 16) run(k_conv_dw_tc<16>, dw_tc_smem<16>());
  if (Cout == 32) run(k_conv_dw_tc<32>, dw_tc_smem<32>());
  if (Cout == 64) run(k_conv_dw_tc<64>, dw_tc_smem<64>());
  if (r) return r;
  k_dw_reduce_tc<<<grid_of(27LL * Cin * Cout), 256, 0, s>>>(part, (int)nblk, tiles, Cin, Cout, dW);
  launch_db(dout, nvox, Cout, work, db, s);
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
