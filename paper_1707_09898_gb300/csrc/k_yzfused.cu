// The y transform fused with the direct z sum, so that the y spectra of the design
// planes never travel through memory.
//
// After the x transform the convolution of Sec. "Discretization", Eq.
// (convolution) is, per column (kx, ky), a 1-D convolution along z with the
// tensor transformed along x and y only (see k_zdir.cu). When the target
// occupies few planes:
//   forward:  out(kx, ky, zo) = sum_z s(kx, ky, zo - z) Y(kx, ky, z), where Y is the
//             y transform of the x-transformed design plane z. k_yz_fwd transforms
//             each design plane of its chunk of z in shared memory and accumulates
//             s Y in registers; k_yz_reduce sums the chunks in a fixed order.
//   adjoint:  Y(kx, ky, z) = sum_p s(kx, ky, z - zp) src(kx, ky, zp) for every design
//             plane z, followed by the inverse y transform: k_zy_adj computes Y in
//             the loader of the inverse transform and writes the real-y rows.
// Same discrete convolution as the unfused passes, without the round trip of the
// y spectra of all design planes through HBM.
#include <cuda.h>  // CUtensorMap and its enums (the encoder is taken from the driver at run time)

#include "fft.cuh"
#include "internal.h"
#include "tma.cuh"

namespace tmk {

namespace {

// s = a - i b for (o, i) at offset dz of column (kx, ky); t points at Tz + kyf*P + kx
__device__ __forceinline__ void tensor_s(const float* t, long long Tc, long long Tdz, float sy, int dz,
                                         const float* coef, int need, float& a, float& b) {
  const int adz = dz < 0 ? -dz : dz;
  const float sz = dz < 0 ? -1.0f : 1.0f;
  const float* p = t + adz * Tdz;
  a = 0.0f;
  b = 0.0f;
  if (need & 1) a += coef[0] * p[0];
  if (need & 2) a += coef[1] * p[Tc];
  if (need & 4) a += coef[2] * p[2 * Tc];
  if (need & 8) a += coef[3] * sy * p[3 * Tc];
  if (need & 16) b += coef[4] * sz * p[4 * Tc];
  if (need & 32) b += coef[5] * sy * sz * p[5 * Tc];
}

// SIMPLE: one input, one source plane, one tensor component c (its sign under y and z
// reflection folded in), so each element is one source load and one tensor load with no
// loop: all loads of a thread are in flight together.
template <int L, bool SIMPLE>
__global__ void __launch_bounds__(kNT, 2) k_zy_adj(ZYArgs a, int c) {
  constexpr int S = plan_stages(L);
  extern __shared__ __align__(16) unsigned char smem[];
  cx<float>* tw = reinterpret_cast<cx<float>*>(smem);
  cx<float>* tile = tw + L;
  load_twiddles<float, kNT>(tw, reinterpret_cast<const cx<float>*>(a.tw), L);
  const int kx0 = blockIdx.x * TB;
  const int z = a.zout0 + blockIdx.y;
  const int o = blockIdx.z;
  const cx<float>* src = reinterpret_cast<const cx<float>*>(a.src);
  cx<float>* out = reinterpret_cast<cx<float>*>(a.out) + a.out_slot[o] * a.out_cstride + z * a.out_zstride + kx0;
  __syncthreads();
  if constexpr (SIMPLE) {
    // first inverse stage (radix R, M = 1) with the direct z sum in its loads: the
    // positions g R + q of a group hold ky = k(g R) + q L/R, so no per-element
    // digit reversal; sign of the folded tensor and of odd dz precomputed
    constexpr int s = S - 1;
    using SS = StageShape<L, s>;
    constexpr int R = SS::R, ITER = (SS::NU + kNT - 1) / kNT;
    const int dz = z - a.zin0;
    const int adz = dz < 0 ? -dz : dz;
    const float cz = (c >= 4 && dz < 0) ? -a.coef[o][0][c] : a.coef[o][0][c];
    const float* tcol = a.Tz + c * a.Tc + adz * a.Tdz + kx0;
    const cx<float>* srow = src + a.in_slot[0] * a.src_cstride + a.zin0 * a.src_zstride + kx0;
    cx<float> v[ITER][R];
#pragma unroll
    for (int it = 0; it < ITER; it++) {
      const int u = it * kNT + threadIdx.x;
      if (SS::NU % kNT == 0 || u < SS::NU) {
        const int line = u % TB, g = u / TB;
        const int kb = k_of_group<L>(g);
#pragma unroll
        for (int q = 0; q < R; q++) {
          const int ky = kb + q * (L / R);
          const bool lo = ky <= L / 2;
          const cx<float> vv = srow[(g * R + q) * a.P + line];
          float f = cz * tcol[(lo ? ky : L - ky) * a.P + line];
          if ((c == 3 || c == 5) && !lo) f = -f;
          v[it][q] = c >= 4 ? mk(f * vv.y, -f * vv.x) : mk(f * vv.x, f * vv.y);  // (-i f) v for xz, yz
        }
      }
    }
#pragma unroll
    for (int it = 0; it < ITER; it++) {
      const int u = it * kNT + threadIdx.x;
      if (SS::NU % kNT == 0 || u < SS::NU) {
        const int line = u % TB, g = u / TB;
        Dft<float, R, true>::run(v[it]);
#pragma unroll
        for (int q = 0; q < R; q++) tile[tidx<false>(g * R + q, line)] = v[it][q];
      }
    }
  } else {
    dit_last_load<float, L, kNT>(tile, [&](int pos, int line) {
      const int ky = k_of_pos<L>(pos);
      const bool lo = ky <= L / 2;
      const int kyf = lo ? ky : L - ky;
      const float sy = lo ? 1.0f : -1.0f;
      const int kx = kx0 + line;
      const float* t = a.Tz + kyf * (long long)a.P + kx;
      const long long so = (long long)pos * a.P + kx;
      cx<float> acc = zero<float>();
      for (int p = 0; p < a.nzin; p++) {
        const int zp = a.zin0 + p;
        for (int i = 0; i < a.nin; i++) {
          const cx<float> v = src[a.in_slot[i] * a.src_cstride + zp * a.src_zstride + so];
          float sa, sb;
          tensor_s(t, a.Tc, a.Tdz, sy, z - zp, a.coef[o][i], a.need[o][i], sa, sb);
          acc = acc + mk(sa * v.x + sb * v.y, sa * v.y - sb * v.x);
        }
      }
      return acc;
    });
  }
  __syncthreads();
  DitRange<float, L, kNT, 1, S - 1>::run(tile, tw);
  dit_stage0_store<float, L, kNT>(tile, tw, [&](int pos, int line, cx<float> v) {
    if (pos < a.n_out) out[(long long)pos * a.P + line] = v;
  });
}

// Forward: one output plane, one output; block (chunk of kx, chunk of z planes) of
// NTF threads (twice the FFT kernels' block: half the sums per thread, twice the warps).
constexpr int NTF = 2 * kNT;
template <int L, bool SIMPLE>
__global__ void __launch_bounds__(NTF, 1) k_yz_fwd(YZArgs a, int c) {
  constexpr int S = plan_stages(L);
  using SL = StageShape<L, S - 1>;
  constexpr int R = SL::R, ITER = (SL::NU + NTF - 1) / NTF;
  extern __shared__ __align__(16) unsigned char smem[];
  cx<float>* tw = reinterpret_cast<cx<float>*>(smem);
  cx<float>* tile = tw + L;
  load_twiddles<float, NTF>(tw, reinterpret_cast<const cx<float>*>(a.tw), L);
  const int kx0 = blockIdx.x * TB;
  const int zb0 = a.zin0 + blockIdx.y * a.zchunk;
  const int zb1 = min(zb0 + a.zchunk, a.zin0 + a.nzin);
  cx<float> acc[ITER][R];
#pragma unroll
  for (int it = 0; it < ITER; it++)
#pragma unroll
    for (int q = 0; q < R; q++) acc[it][q] = zero<float>();
  const cx<float>* in0 = reinterpret_cast<const cx<float>*>(a.in);
  for (int z = zb0; z < zb1; z++) {
    for (int i = 0; i < (SIMPLE ? 1 : a.nin); i++) {
      const cx<float>* in = in0 + a.in_slot[i] * a.in_cstride + z * a.in_zstride + kx0;
      __syncthreads();
      dif_stage0_load<float, L, NTF>(tile, tw, [&](int pos, int line) {
        return pos < a.n_in ? in[(long long)pos * a.P + line] : zero<float>();
      });
      __syncthreads();
      DifRange<float, L, NTF, 1, S - 1>::run(tile, tw);
      // last stage in registers, then s(zo - z) times the spectrum into the sums
      const int dz = a.zout - z;
#pragma unroll
      for (int it = 0; it < ITER; it++) {
        const int u = it * NTF + threadIdx.x;
        if (SL::NU % NTF == 0 || u < SL::NU) {
          const int line = u % TB, g = u / TB;
          cx<float> v[R];
#pragma unroll
          for (int q = 0; q < R; q++) v[q] = tile[tidx<false>(g * R + q, line)];
          Dft<float, R, false>::run(v);
          const int kb = k_of_group<L>(g);
          const int kx = kx0 + line;
#pragma unroll
          for (int q = 0; q < R; q++) {
            const int ky = kb + q * (L / R);
            const bool lo = ky <= L / 2;
            const float* t = a.Tz + (lo ? ky : L - ky) * (long long)a.P + kx;
            if constexpr (SIMPLE) {
              const int adz = dz < 0 ? -dz : dz;
              float f = a.coef[0][c] * t[c * a.Tc + adz * a.Tdz];
              if ((c == 3 || c == 5) && !lo) f = -f;
              if (c >= 4 && dz < 0) f = -f;
              acc[it][q] = acc[it][q] + (c >= 4 ? mk(f * v[q].y, -f * v[q].x) : mk(f * v[q].x, f * v[q].y));
            } else {
              float sa, sb;
              tensor_s(t, a.Tc, a.Tdz, lo ? 1.0f : -1.0f, dz, a.coef[i], a.need[i], sa, sb);
              acc[it][q] = acc[it][q] + mk(sa * v[q].x + sb * v[q].y, sa * v[q].y - sb * v[q].x);
            }
          }
        }
      }
    }
  }
  // partial of this z chunk, at the spectrum's positions
  cx<float>* part = reinterpret_cast<cx<float>*>(a.part) + (long long)blockIdx.y * L * a.P + kx0;
#pragma unroll
  for (int it = 0; it < ITER; it++) {
    const int u = it * NTF + threadIdx.x;
    if (SL::NU % NTF == 0 || u < SL::NU) {
      const int line = u % TB, g = u / TB;
#pragma unroll
      for (int q = 0; q < R; q++) part[(long long)(g * R + q) * a.P + line] = acc[it][q];
    }
  }
}


// The single-component forward with the next design plane's input rows and tensor
// slice copied into shared memory (cp.async, two buffers) while the current plane is
// transformed, so the loads overlap the transform instead of following it.
__device__ __forceinline__ void cp16(void* sdst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }


template <int L>
__global__ void __launch_bounds__(NTF, 1) k_yz_fwd_staged(YZArgs a, int c) {
  constexpr int S = plan_stages(L);
  using SL = StageShape<L, S - 1>;
  constexpr int R = SL::R, ITER = (SL::NU + NTF - 1) / NTF;
  constexpr int KY = L / 2 + 1;
  extern __shared__ __align__(16) unsigned char smem[];
  cx<float>* tw = reinterpret_cast<cx<float>*>(smem);
  cx<float>* tile = tw + L;
  cx<float>* sin0 = tile + L * TB;                               // [2][L/2][TB] input rows
  float* st0 = reinterpret_cast<float*>(sin0 + 2 * (L / 2) * TB);  // [2][KY][TB] tensor slice
  load_twiddles<float, NTF>(tw, reinterpret_cast<const cx<float>*>(a.tw), L);
  const int kx0 = blockIdx.x * TB;
  const int zb0 = a.zin0 + blockIdx.y * a.zchunk;
  const int zb1 = min(zb0 + a.zchunk, a.zin0 + a.nzin);
  const cx<float>* in0 = reinterpret_cast<const cx<float>*>(a.in) + a.in_slot[0] * a.in_cstride + kx0;
  const float* tc = a.Tz + c * a.Tc + kx0;
  auto issue = [&](int z, int buf) {  // 16-byte copies: 8 per input row, 4 per tensor row
    const cx<float>* src = in0 + z * a.in_zstride;
    cx<float>* sin = sin0 + buf * (L / 2) * TB;
    for (int q = threadIdx.x; q < a.n_in * 8; q += NTF) {
      const int row = q >> 3, part = q & 7;
      cp16(sin + row * TB + part * 2, src + (long long)row * a.P + part * 2);
    }
    const int dz = a.zout - z, adz = dz < 0 ? -dz : dz;
    const float* t = tc + adz * a.Tdz;
    float* stt = st0 + buf * KY * TB;
    for (int q = threadIdx.x; q < KY * 4; q += NTF) {
      const int row = q >> 2, part = q & 3;
      cp16(stt + row * TB + part * 4, t + (long long)row * a.P + part * 4);
    }
    cp_commit();
  };
  cx<float> acc[ITER][R];
#pragma unroll
  for (int it = 0; it < ITER; it++)
#pragma unroll
    for (int q = 0; q < R; q++) acc[it][q] = zero<float>();
  if (zb0 < zb1) issue(zb0, 0);
  for (int z = zb0; z < zb1; z++) {
    const int buf = (z - zb0) & 1;
    __syncthreads();  // every thread is done with the other buffer and with the tile
    if (z + 1 < zb1) {
      issue(z + 1, buf ^ 1);
      cp_wait<1>();
    } else {
      cp_wait<0>();
    }
    __syncthreads();  // plane z's copies of every thread have landed
    const cx<float>* sin = sin0 + buf * (L / 2) * TB;
    const float* stt = st0 + buf * KY * TB;
    dif_stage0_load<float, L, NTF>(tile, tw, [&](int pos, int line) {
      return pos < a.n_in ? sin[pos * TB + line] : zero<float>();
    });
    __syncthreads();
    DifRange<float, L, NTF, 1, S - 1>::run(tile, tw);
    const int dz = a.zout - z;
    const float cz = (c >= 4 && dz < 0) ? -a.coef[0][c] : a.coef[0][c];
#pragma unroll
    for (int it = 0; it < ITER; it++) {
      const int u = it * NTF + threadIdx.x;
      if (SL::NU % NTF == 0 || u < SL::NU) {
        const int line = u % TB, g = u / TB;
        cx<float> v[R];
#pragma unroll
        for (int q = 0; q < R; q++) v[q] = tile[tidx<false>(g * R + q, line)];
        Dft<float, R, false>::run(v);
        const int kb = k_of_group<L>(g);
#pragma unroll
        for (int q = 0; q < R; q++) {
          const int ky = kb + q * (L / R);
          const bool lo = ky <= L / 2;
          float f = cz * stt[(lo ? ky : L - ky) * TB + line];
          if ((c == 3 || c == 5) && !lo) f = -f;
          acc[it][q] = acc[it][q] + (c >= 4 ? mk(f * v[q].y, -f * v[q].x) : mk(f * v[q].x, f * v[q].y));
        }
      }
    }
  }
  cx<float>* part = reinterpret_cast<cx<float>*>(a.part) + (long long)blockIdx.y * L * a.P + kx0;
#pragma unroll
  for (int it = 0; it < ITER; it++) {
    const int u = it * NTF + threadIdx.x;
    if (SL::NU % NTF == 0 || u < SL::NU) {
      const int line = u % TB, g = u / TB;
#pragma unroll
      for (int q = 0; q < R; q++) part[(long long)(g * R + q) * a.P + line] = acc[it][q];
    }
  }
}

// ---------------------------------------------------------------------------
// Warp-specialized versions of the two single-component kernels for two-stage plans
// whose first stage has kNT units and whose last stage has 2 kNT (L = 512 = 32 x 16): a
// block of 512 threads runs two groups of eight warps on one plane each, a plane apart,
// with a tile per group and one block barrier per plane:
//   forward: the "transform" warps take the input rows of plane z + 1 (loaded into
//            registers a round ahead) and run the first DIF stage into one tile while
//            the "accumulate" warps finish plane z from the other tile (the last stage
//            in registers) and add s(zo - z) times it into their sums;
//   adjoint: the "load" warps form s(z - zp) times the source spectrum (held in
//            registers per column block) for plane z + 1 and run the first inverse
//            stage into one tile while the "store" warps finish plane z from the other
//            tile and write its rows.
// The (column block, plane) items are spread evenly over one block per SM, z fastest;
// each block follows its item's column block and plane by increments (no divisions in
// the loop). The tensor slices arrive in shared memory by TMA (two boxes per slice,
// mbarrier completion) a round ahead, from a copy of the one tensor component C with
// the coupling coefficient already multiplied in (s = coef N^_C, the same float32
// products as multiplying in the kernel). C fixes the sign rules of the folded tensor at
// compile time; the positions of the last stage are g R1 + q with frequency
// ky = g + q L/R1, so the tensor row of every element is a compile-time offset from one
// of two per-thread bases. The first stage of the forward transform skips the zero
// half of its inputs (rows y >= L/2) and the last stage of the inverse computes only
// the rows y < L/2 it keeps; both stages' radix-2 butterflies run in fused
// multiply-adds (DftF). FULL: every row y < L/2 is valid (n = L/2), no predicates.
template <int L>
__host__ __device__ constexpr bool yz_ws_plan() {
  return plan_stages(L) == 2 && StageShape<L, 0>::NU == kNT && StageShape<L, 1>::NU == 2 * kNT &&
         StageShape<L, 0>::R == 2 * TB && StageShape<L, 0>::M == TB && StageShape<L, 1>::R == TB;
}

constexpr int kBarAll = 1, kBarGroup = 2;  // named barriers (0 is __syncthreads)

// tensor factor of last-stage element q of group g from the scaled slice, with C's sign
// rules: odd in ky for xy and yz (C = 3, 5), odd in dz for xz and yz (C = 4, 5; neg means
// dz < 0); tlo = slice + g TB + line (rows g + q L/R1), thi = slice + (L - g) TB + line
template <int L, int C>
__device__ __forceinline__ float ws_tensor(const float* tlo, const float* thi, int g, int q, bool neg) {
  constexpr int R1 = StageShape<L, 1>::R, QS = L / R1;
  const float f = q < R1 / 2 ? tlo[q * QS * TB] : thi[-q * QS * TB];
  bool flip = C >= 4 && neg;
  // ky = g + q QS lies above L/2 for q > R1/2, and for q = R1/2 unless g = 0
  if constexpr (C == 3 || C == 5) {
    if (q > R1 / 2 || (q == R1 / 2 && g > 0)) flip = !flip;
  }
  return flip ? -f : f;
}
template <int C>
__device__ __forceinline__ cx<float> ws_apply(float f, cx<float> v) {  // (-i f) v for xz, yz
  return C >= 4 ? mk(f * v.y, -f * v.x) : mk(f * v.x, f * v.y);
}

// The stage-0 twiddle of position j + q M0 (= g R1 + q' with j = q', q = g) is W^(j q),
// applied after the first DIF stage or before the last DIT stage, by either group: in the
// forward all of it by the accumulate warps (their stage-0 partners set the pace: moving
// the work the other way cost 8 us per launch), in the adjoint shared, q < R0/2 by the
// store warps and the rest by the load warps (their second unit, g >= R0/2); the other
// splits measured no faster there.
// TW: 0 = q < R0/2 here (the rest by the other group), 1 = all, 2 = none
template <int L, bool INV, int TW>
__device__ __forceinline__ void twiddles_lo(cx<float>* v, int j, const cx<float>* tw) {
  constexpr int R0 = StageShape<L, 0>::R;
  if (TW == 2 || j == 0) return;
#pragma unroll
  for (int q = 1; q < (TW == 1 ? R0 : R0 / 2); q++) v[q] = INV ? cmulc(v[q], tw[j * q]) : cmul(v[q], tw[j * q]);
}
constexpr int kFwdTw = 2, kAdjTw = 0;
template <int L, bool INV>
__device__ __forceinline__ void twiddles_hi(cx<float>* v, int g, const cx<float>* tw) {
  constexpr int R1 = StageShape<L, 1>::R;
#pragma unroll
  for (int q = 1; q < R1; q++) v[q] = INV ? cmulc(v[q], tw[q * g]) : cmul(v[q], tw[q * g]);
}

// Tensor slices: L/2 + 1 rows of TB floats, fetched as two TMA boxes of KB = L/4 + 2 rows
// (the rows past L/2 are not used); KB is even, so both box destinations (KB TB floats
// apart) stay on 128-byte boundaries
template <int L>
__host__ __device__ constexpr int slice_box_rows() {
  return L / 4 + 2;
}
template <int L>
__host__ __device__ constexpr int slice_rows() {
  return 2 * slice_box_rows<L>();
}
static_assert((slice_box_rows<512>() * TB * sizeof(float)) % 128 == 0, "128-byte aligned TMA destinations");
static_assert((512 + 2 * 512 * TB) * sizeof(float2) % 128 == 0, "128-byte aligned TMA destinations");
// 128 bytes of slack to align the dynamic buffer for the TMA destinations; mbarriers last
template <int L>
constexpr size_t ws_smem() {
  return 128 + (size_t)(L + 2 * L * TB) * sizeof(float2) + (size_t)2 * slice_rows<L>() * TB * sizeof(float) +
         2 * sizeof(unsigned long long);
}

// (column block, plane) of an item index i, planes z0 .. z0 + nz - 1 per column block,
// and the step to the next item
struct Item {
  int cb, z;
};
__device__ __forceinline__ Item item_of(long long i, int z0, int nz) {
  const int cb = (int)(i / nz);
  return {cb, z0 + (int)(i - (long long)cb * nz)};
}
__device__ __forceinline__ Item next_item(Item it, int z0, int nz) {
  return it.z + 1 == z0 + nz ? Item{it.cb + 1, z0} : Item{it.cb, it.z + 1};
}

// Forward, flattened: block b transforms the (column block, design plane) items
// [T b / B, T (b + 1) / B), T = (P / TB) nzin. The sums of a column block are written as
// a segment partial after the block's last item of it (at most two segments per block,
// as long as B >= P / TB); k_yz_finish adds the segments of each column block in block
// order and runs the target plane's inverse y transform.
template <int L, int C, bool FULL>
__global__ void __launch_bounds__(NTF, 1) k_yz_fwd_ws(YZArgs a, const __grid_constant__ CUtensorMap mslice) {
  using S0 = StageShape<L, 0>;
  using S1 = StageShape<L, 1>;
  constexpr int R0 = S0::R, M0 = S0::M, R1 = S1::R, KS = slice_rows<L>(), KB = slice_box_rows<L>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);  // TMA destinations
  cx<float>* tw = reinterpret_cast<cx<float>*>(smem);
  cx<float>* tiles = tw + L;                                      // [2][L][TB]
  float* stt0 = reinterpret_cast<float*>(tiles + 2 * L * TB);     // [2][KS][TB] tensor slices
  unsigned long long* mb = reinterpret_cast<unsigned long long*>(stt0 + 2 * KS * TB);  // slice 0, slice 1
  load_twiddles<float, NTF>(tw, reinterpret_cast<const cx<float>*>(a.tw), L);
  if (threadIdx.x == 0) {
    mbar_init(mb, 1);
    mbar_init(mb + 1, 1);
    mbar_init_fence();
  }
  pdl_wait();  // the x spectra and the segment buffer belong to earlier kernels
  const long long T = (long long)(a.P / TB) * a.nzin;
  const long long i0 = T * blockIdx.x / gridDim.x, i1 = T * (blockIdx.x + 1) / gridDim.x;
  const int n = (int)(i1 - i0);
  const Item first = item_of(i0, a.zin0, a.nzin);
  __syncthreads();
  if (threadIdx.x < kNT) {
    // transform warps: stage 0 of item i0 + r in round r, its 16 input values per thread
    // loaded into registers a round ahead; thread 0 issues the TMA copy of the item's
    // tensor slice, which the accumulate warps use in the next round
    const int t = threadIdx.x;
    const int line = t % TB, j = t / TB;
    const cx<float>* in0 =
        reinterpret_cast<const cx<float>*>(a.in) + a.in_slot[0] * a.in_cstride + (long long)j * a.P + line;
    cx<float> pre[R0 / 2];  // rows j + q M0 (q < R0/2; n_in <= L/2) of the next item
    auto fetch = [&](Item it) {
      const cx<float>* src = in0 + it.z * a.in_zstride + it.cb * TB;
#pragma unroll
      for (int q = 0; q < R0 / 2; q++)
        pre[q] = (FULL || j + q * M0 < a.n_in) ? src[(long long)q * M0 * a.P] : zero<float>();
    };
    auto issue_slice = [&](Item it, int buf) {
      const int dz = a.zout - it.z, adz = dz < 0 ? -dz : dz;
      float* stt = stt0 + buf * KS * TB;
      mbar_expect_tx(mb + buf, 2 * KB * TB * (int)sizeof(float));
      tma_load_2d(stt, &mslice, it.cb * TB, adz * (L / 2 + 1), mb + buf);
      tma_load_2d(stt + KB * TB, &mslice, it.cb * TB, adz * (L / 2 + 1) + KB, mb + buf);
    };
    Item cur = first;
    if (n > 0) fetch(cur);
    for (int r = 0; r <= n; r++) {
      if (r < n) {
        cx<float> v[R0];
#pragma unroll
        for (int q = 0; q < R0 / 2; q++) v[q] = pre[q];
        const Item nxt = next_item(cur, a.zin0, a.nzin);
        if (r + 1 < n) fetch(nxt);
        if (t == 0) {
          if (r == 0) fence_proxy_async_global();  // the scaled tensor was written by ordinary stores
          fence_proxy_async_smem();  // the other group read this slice buffer a round ago
          issue_slice(cur, r & 1);
        }
        cur = nxt;
        dft32_half_input<false>(v);
        twiddles_lo<L, false, kFwdTw>(v, j, tw);  // none here: the accumulate warps apply them
        cx<float>* tile = tiles + (r & 1) * L * TB;
#pragma unroll
        for (int q = 0; q < R0; q++) tile[(j + q * M0) * TB + line] = v[q];
      }
      bar_named(kBarAll, NTF);
    }
  } else {
    // accumulate warps: last stage of item i0 + r - 1 in round r, times s, into the sums
    const int t = threadIdx.x - kNT;
    cx<float> acc[2][R1];
#pragma unroll
    for (int it = 0; it < 2; it++)
#pragma unroll
      for (int q = 0; q < R1; q++) acc[it][q] = zero<float>();
    Item cur = first;  // the item of the next round
    for (int r = 0; r <= n; r++) {
      if (r >= 1) {
        const bool neg = a.zout - cur.z < 0;
        const cx<float>* tile = tiles + ((r - 1) & 1) * L * TB;
        const float* stt = stt0 + ((r - 1) & 1) * KS * TB;
        mbar_wait(mb + ((r - 1) & 1), ((r - 1) >> 1) & 1, a.status);  // its tensor slice
#pragma unroll
        for (int it = 0; it < 2; it++) {
          const int u = it * kNT + t, line = u % TB, g = u / TB;
          cx<float> v[R1];
#pragma unroll
          for (int q = 0; q < R1; q++) v[q] = tile[(g * R1 + q) * TB + line];
          if (kFwdTw == 2 || (kFwdTw == 0 && it == 1)) twiddles_hi<L, false>(v, g, tw);  // stage-0 twiddles
          DftF<R1, false>::run(v);
          const float* tlo = stt + g * TB + line;
          const float* thi = stt + (L - g) * TB + line;
#pragma unroll
          for (int q = 0; q < R1; q++) acc[it][q] = acc[it][q] + ws_apply<C>(ws_tensor<L, C>(tlo, thi, g, q, neg), v[q]);
        }
        const bool last = cur.z + 1 == a.zin0 + a.nzin;  // the last plane of column block cur.cb
        if (r == n || last) {  // the block's last item of column block cur.cb
          const int sg = cur.cb == first.cb ? 0 : 1;
          cx<float>* seg = reinterpret_cast<cx<float>*>(a.seg) + (long long)(blockIdx.x * 2 + sg) * L * TB;
#pragma unroll
          for (int it = 0; it < 2; it++) {
            const int u = it * kNT + t, line = u % TB, g = u / TB;
#pragma unroll
            for (int q = 0; q < R1; q++) {
              seg[(g * R1 + q) * TB + line] = acc[it][q];
              acc[it][q] = zero<float>();
            }
          }
        }
        cur = next_item(cur, a.zin0, a.nzin);
      }
      bar_named(kBarAll, NTF);
    }
  }
}

// The target plane after the forward: for column block cb (blockIdx.x), the segment
// partials of the blocks that held its items, added in block order, then its inverse y
// transform (the inverse of the two DIF stages) into rows y < n_in of A. Each block takes
// FL of the column block's TB lines (blockIdx.y). The segments of a column block are read
// kFinishSegs at a time with all their loads in flight (the sums are latency-bound: a few
// megabytes from L2 spread over the column blocks).
constexpr int kFinishLines = 2, kFinishThreads = 512, kFinishSegs = 12, kFinishMaxBlocks = 1024;
// tile slot of (pos, line) in the finishing kernel: positions XOR-swizzled by pos / 16 so that
// the threads of a stage (consecutive groups g at one q, or consecutive j) hit distinct banks
__device__ __forceinline__ int fin_idx(int pos, int l) { return (pos ^ ((pos >> 4) & 15)) * kFinishLines + l; }
template <int L>
__global__ void __launch_bounds__(kFinishThreads) k_yz_finish(YZArgs a, int B) {
  using S0 = StageShape<L, 0>;
  using S1 = StageShape<L, 1>;
  constexpr int R0 = S0::R, M0 = S0::M, R1 = S1::R, FL = kFinishLines, NT = kFinishThreads, NE = L * FL / NT;
  static_assert(NE * NT == L * FL, "elements per thread");
  __shared__ cx<float> tw[L];
  __shared__ cx<float> tile[L * FL];
  __shared__ int segidx[kFinishMaxBlocks];
  load_twiddles<float, NT>(tw, reinterpret_cast<const cx<float>*>(a.tw), L);
  const int cb = blockIdx.x, l0 = blockIdx.y * FL;
  const long long T = (long long)(a.P / TB) * a.nzin;
  const long long x0 = (long long)cb * a.nzin, x1 = x0 + a.nzin - 1;  // first and last item of cb
  const int b_lo = (int)(((x0 + 1) * B - 1) / T), b_hi = (int)(((x1 + 1) * B - 1) / T);
  const int nseg = b_hi - b_lo + 1;
  // segment of block b holding column block cb: its first (0) or its second (1)
  for (int k = threadIdx.x; k < nseg; k += NT) {
    const int b = b_lo + k;
    segidx[k] = 2 * b + ((int)((T * b / B) / a.nzin) == cb ? 0 : 1);
  }
  pdl_wait();  // the segment partials come from the forward kernel
  __syncthreads();
  const cx<float>* segs = reinterpret_cast<const cx<float>*>(a.seg) + l0;
  int off[NE];
#pragma unroll
  for (int k = 0; k < NE; k++) {
    const int e = threadIdx.x + NT * k;
    off[k] = (e / FL) * TB + e % FL;
  }
  cx<float> acc[NE];
#pragma unroll
  for (int k = 0; k < NE; k++) acc[k] = zero<float>();
  for (int s0 = 0; s0 < nseg; s0 += kFinishSegs) {
    cx<float> v[kFinishSegs][NE];
#pragma unroll
    for (int s = 0; s < kFinishSegs; s++) {
      if (s0 + s < nseg) {
        const cx<float>* sp = segs + (long long)segidx[s0 + s] * L * TB;
#pragma unroll
        for (int k = 0; k < NE; k++) {
          const float2 t = __ldcg(reinterpret_cast<const float2*>(sp + off[k]));
          v[s][k] = mk(t.x, t.y);
        }
      }
    }
#pragma unroll
    for (int s = 0; s < kFinishSegs; s++)
      if (s0 + s < nseg)
#pragma unroll
        for (int k = 0; k < NE; k++) acc[k] = acc[k] + v[s][k];
  }
#pragma unroll
  for (int k = 0; k < NE; k++) {
    const int e = threadIdx.x + NT * k;
    tile[fin_idx(e / FL, e % FL)] = acc[k];
  }
  __syncthreads();
  if (threadIdx.x < (L / R1) * FL) {  // first inverse stage: groups g, positions g R1 + q
    const int g = threadIdx.x / FL, l = threadIdx.x % FL;
    cx<float> v[R1];
#pragma unroll
    for (int q = 0; q < R1; q++) v[q] = tile[fin_idx(g * R1 + q, l)];
    DftF<R1, true>::run(v);
#pragma unroll
    for (int q = 0; q < R1; q++) tile[fin_idx(g * R1 + q, l)] = v[q];
  }
  __syncthreads();
  if (threadIdx.x < M0 * FL) {  // last inverse stage (plan stage 0): rows y = j + q M0 < n_in
    const int j = threadIdx.x / FL, l = threadIdx.x % FL;
    cx<float> v[R0];
#pragma unroll
    for (int q = 0; q < R0; q++) v[q] = tile[fin_idx(j + q * M0, l)];
    apply_twiddles<float, L, 0, true>(v, j, tw);
    cx<float>* o = reinterpret_cast<cx<float>*>(a.yrows) + cb * TB + l0 + l;
    if (a.n_in <= L / 2) {  // the kept rows y = j + q M0 < n_in have q < R0/2
      dft_low_half<R0, true>(v);
#pragma unroll
      for (int q = 0; q < R0 / 2; q++) {
        const int y = j + q * M0;
        if (y < a.n_in) o[(long long)y * a.P] = v[q];
      }
    } else {
      DftF<R0, true>::run(v);
#pragma unroll
      for (int q = 0; q < R0; q++) {
        const int y = j + q * M0;
        if (y < a.n_in) o[(long long)y * a.P] = v[q];
      }
    }
  }
}

// Adjoint: the (column block, design plane) items [T b / B, T (b + 1) / B) of block b,
// T = (P / TB) nzout; one item per round and group.
template <int L, int C, bool FULL>
__global__ void __launch_bounds__(NTF, 1) k_zy_adj_ws(ZYArgs a, const __grid_constant__ CUtensorMap mslice) {
  using S0 = StageShape<L, 0>;
  using S1 = StageShape<L, 1>;
  constexpr int R0 = S0::R, M0 = S0::M, R1 = S1::R, KS = slice_rows<L>(), KB = slice_box_rows<L>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);  // TMA destinations
  cx<float>* tw = reinterpret_cast<cx<float>*>(smem);
  cx<float>* tiles = tw + L;                                      // [2][L][TB]
  float* stt0 = reinterpret_cast<float*>(tiles + 2 * L * TB);     // [2][KS][TB] tensor slices
  unsigned long long* mb = reinterpret_cast<unsigned long long*>(stt0 + 2 * KS * TB);  // slice 0, slice 1
  load_twiddles<float, NTF>(tw, reinterpret_cast<const cx<float>*>(a.tw), L);
  const long long T = (long long)(a.P / TB) * a.nzout;
  const long long i0 = T * blockIdx.x / gridDim.x, i1 = T * (blockIdx.x + 1) / gridDim.x;
  const int n = (int)(i1 - i0);
  const Item first = item_of(i0, a.zout0, a.nzout);
  auto issue_slice = [&](Item it, int buf) {  // one thread: two TMA boxes into slice buffer buf
    const int dz = it.z - a.zin0, adz = dz < 0 ? -dz : dz;
    float* stt = stt0 + buf * KS * TB;
    mbar_expect_tx(mb + buf, 2 * KB * TB * (int)sizeof(float));
    tma_load_2d(stt, &mslice, it.cb * TB, adz * (L / 2 + 1), mb + buf);
    tma_load_2d(stt + KB * TB, &mslice, it.cb * TB, adz * (L / 2 + 1) + KB, mb + buf);
  };
  if (threadIdx.x == 0) {
    mbar_init(mb, 1);
    mbar_init(mb + 1, 1);
    mbar_init_fence();
    fence_proxy_async_global();  // the scaled tensor was written by ordinary stores
    if (n > 0) issue_slice(first, 0);  // the tensor is constant: no need to wait for earlier kernels
  }
  pdl_wait();  // the source plane and the outputs belong to earlier kernels
  if (a.zero_word && blockIdx.x == 0 && threadIdx.x == 0) *a.zero_word = 0u;
  __syncthreads();
  if (threadIdx.x < kNT) {
    // load warps: s times the source, first inverse stage, into tile r % 2 in round r
    const int t = threadIdx.x;
    const cx<float>* src = reinterpret_cast<const cx<float>*>(a.src) + a.in_slot[0] * a.src_cstride +
                           a.zin0 * a.src_zstride;
    // the source spectrum does not depend on the design plane: a thread keeps its 2 R1
    // values (positions g R1 + q of its two units) for as long as the column block stays
    cx<float> sv[2][R1];
    int cb_held = -1;
    Item cur = first;
    for (int r = 0; r <= n; r++) {
      if (r < n) {
        if (cur.cb != cb_held) {
          if (a.gsrc) {
            // the forward y transform of the source's column block, here: rows y < n_src of
            // the x-transformed source plane through the first DIF stage into this round's
            // tile (the store warps work on the other one), the second stage into registers
            cx<float>* scr = tiles + (r & 1) * L * TB;
            {
              const int line = t % TB, j = t / TB;
              const cx<float>* g0 = reinterpret_cast<const cx<float>*>(a.gsrc) + (long long)j * a.P + cur.cb * TB + line;
              cx<float> v[R0];
#pragma unroll
              for (int q = 0; q < R0 / 2; q++) v[q] = j + q * M0 < a.n_src ? g0[(long long)q * M0 * a.P] : zero<float>();
              dft32_half_input<false>(v);
              if (j != 0) {
#pragma unroll
                for (int q = 1; q < R0; q++) v[q] = cmul(v[q], tw[j * q]);
              }
#pragma unroll
              for (int q = 0; q < R0; q++) scr[(j + q * M0) * TB + line] = v[q];
            }
            bar_named(kBarGroup, kNT);
#pragma unroll
            for (int it = 0; it < 2; it++) {
              const int u = it * kNT + t, line = u % TB, g = u / TB;
#pragma unroll
              for (int q = 0; q < R1; q++) sv[it][q] = scr[(g * R1 + q) * TB + line];
              DftF<R1, false>::run(sv[it]);
            }
            bar_named(kBarGroup, kNT);  // the tile is free for this round's first stage
          } else {
#pragma unroll
            for (int it = 0; it < 2; it++) {
              const int u = it * kNT + t, line = u % TB, g = u / TB;
              const cx<float>* s = src + (long long)(g * R1) * a.P + cur.cb * TB + line;
#pragma unroll
              for (int q = 0; q < R1; q++) sv[it][q] = s[q * a.P];
            }
          }
          cb_held = cur.cb;
        }
        const bool neg = cur.z - a.zin0 < 0;
        const float* stt = stt0 + (r & 1) * KS * TB;
        cx<float>* tile = tiles + (r & 1) * L * TB;
        mbar_wait(mb + (r & 1), (r >> 1) & 1, a.status);  // this item's tensor slice
#pragma unroll
        for (int it = 0; it < 2; it++) {
          const int u = it * kNT + t, line = u % TB, g = u / TB;
          const float* tlo = stt + g * TB + line;
          const float* thi = stt + (L - g) * TB + line;
          cx<float> v[R1];
#pragma unroll
          for (int q = 0; q < R1; q++) v[q] = ws_apply<C>(ws_tensor<L, C>(tlo, thi, g, q, neg), sv[it][q]);
          DftF<R1, true>::run(v);
          if (kAdjTw == 2 || (kAdjTw == 0 && it == 1)) twiddles_hi<L, true>(v, g, tw);  // stage-0 twiddles
#pragma unroll
          for (int q = 0; q < R1; q++) tile[(g * R1 + q) * TB + line] = v[q];
        }
        cur = next_item(cur, a.zout0, a.nzout);
      }
      bar_named(kBarAll, NTF);
    }
  } else {
    // store warps: last inverse stage of the item of round r - 1, rows y < n_out out
    const int t = threadIdx.x - kNT;
    const int line = t % TB, j = t / TB;
    cx<float>* out0 = reinterpret_cast<cx<float>*>(a.out) + a.out_slot[0] * a.out_cstride;
    Item cur = first;                                   // the item of round r - 1
    Item ahead = next_item(first, a.zout0, a.nzout);    // the item whose slice is issued in round r
    for (int r = 0; r <= n; r++) {
      if (t == 0 && r + 1 < n) {
        fence_proxy_async_smem();  // the other group read this slice buffer a round ago
        issue_slice(ahead, (r + 1) & 1);
      }
      if (r + 1 < n) ahead = next_item(ahead, a.zout0, a.nzout);
      if (r >= 1) {
        const cx<float>* tile = tiles + ((r - 1) & 1) * L * TB;
        cx<float> v[R0];
#pragma unroll
        for (int q = 0; q < R0; q++) v[q] = tile[(j + q * M0) * TB + line];
        twiddles_lo<L, true, kAdjTw>(v, j, tw);  // else q >= R0/2: applied by the load warps
        cx<float>* o = out0 + cur.z * a.out_zstride + cur.cb * TB + line;
        if constexpr (FULL) {  // rows y = j + q M0 < L/2: the first half of the outputs
          dft_low_half<R0, true>(v);
#pragma unroll
          for (int q = 0; q < R0 / 2; q++) o[(long long)(j + q * M0) * a.P] = v[q];
        } else {
          DftF<R0, true>::run(v);
#pragma unroll
          for (int q = 0; q < R0; q++) {
            const int y = j + q * M0;
            if (y < a.n_out) o[(long long)y * a.P] = v[q];
          }
        }
        cur = next_item(cur, a.zout0, a.nzout);
      }
      bar_named(kBarAll, NTF);
    }
  }
}

// out[pos][kx] = sum over z chunks of the partials, in chunk order
__global__ void k_yz_reduce(const float2* part, int nchunks, long long plane, float2* out) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < plane;
       e += (long long)gridDim.x * blockDim.x) {
    float2 s = part[e];
    for (int c = 1; c < nchunks; c++) {
      const float2 v = part[(long long)c * plane + e];
      s.x += v.x;
      s.y += v.y;
    }
    out[e] = s;
  }
}

template <int L>
size_t fused_smem() {
  return (size_t)(L + L * TB) * sizeof(float2);
}

// the single tensor component of (o, i) = (0, 0), or -1
int single_component(const int need) { return (need != 0 && (need & (need - 1)) == 0) ? __builtin_ctz(need) : -1; }

template <int L, bool SIMPLE>
int launch_adj(const ZYArgs& a, int c, cudaStream_t s) {
  const size_t sm = fused_smem<L>();
  static bool init = false;
  if (!init) {
    if (cudaFuncSetAttribute(k_zy_adj<L, SIMPLE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) !=
        cudaSuccess)
      return -1;
    init = true;
  }
  k_zy_adj<L, SIMPLE><<<dim3(a.P / TB, a.nzout, a.nout), kNT, sm, s>>>(a, c);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

// cuTensorMapEncodeTiled from the driver (no link-time dependency on libcuda)
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encoder() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(f);
  }
  return fn;
}
// 2-D map over a row-major array of `outer` rows of `inner` elements, row pitch `pitch`
// bytes, boxes of box_inner x box_outer elements; false if it cannot be encoded
bool map_2d(CUtensorMap* m, CUtensorMapDataType type, const void* base, unsigned long long inner,
            unsigned long long outer, unsigned long long pitch, unsigned box_inner, unsigned box_outer) {
  EncodeTiledFn fn = encoder();
  if (!fn || (reinterpret_cast<uintptr_t>(base) & 15) || (pitch & 15)) return false;
  const cuuint64_t dims[2] = {inner, outer};
  const cuuint64_t strides[1] = {pitch};
  const cuuint32_t box[2] = {box_inner, box_outer};
  const cuuint32_t es[2] = {1, 1};
  return fn(m, type, 2, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}
// the tensor slices: a scaled single component Ts [nz][Ly/2 + 1][P] floats as rows of P;
// the last two maps made on this host thread are kept (a context launches the forward
// and the adjoint with the same two every time)
bool slice_map(CUtensorMap* m, const float* Ts, long long rows, int P, int box_rows) {
  struct Cached {
    const float* Ts = nullptr;
    long long rows = 0;
    int P = 0, box = 0;
    CUtensorMap map;
  };
  thread_local Cached c[2];
  thread_local int next = 0;
  for (Cached& e : c)
    if (e.Ts == Ts && e.rows == rows && e.P == P && e.box == box_rows) {
      *m = e.map;
      return true;
    }
  if (!map_2d(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, Ts, (unsigned long long)P, (unsigned long long)rows,
              (unsigned long long)P * sizeof(float), TB, box_rows))
    return false;
  Cached& e = c[next];
  next ^= 1;
  e.Ts = Ts;
  e.rows = rows;
  e.P = P;
  e.box = box_rows;
  e.map = *m;
  return true;
}

int sm_count() {
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 148;
  }
  return nsm;
}

template <int L, int C, bool FULL>
int launch_adj_ws(const ZYArgs& a, const CUtensorMap& mslice, cudaStream_t s) {
  constexpr size_t sm = ws_smem<L>();
  static bool init = false;
  if (!init) {
    if (cudaFuncSetAttribute(k_zy_adj_ws<L, C, FULL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) !=
        cudaSuccess)
      return -1;
    init = true;
  }
  const long long items = (long long)(a.P / TB) * a.nzout;
  const int blocks = (int)(items < sm_count() ? items : sm_count());  // one resident block per SM
  return launch_k(k_zy_adj_ws<L, C, FULL>, dim3(blocks), dim3(NTF), sm, s, a.pdl != 0, a, mslice) == cudaSuccess
             ? (a.zero_word ? 1 : 0)  // 1: *zero_word is cleared
             : -1;
}
template <int L, bool FULL>
int launch_adj_ws_c(const ZYArgs& a, int c, const CUtensorMap& ms, cudaStream_t s) {
  switch (c) {
    case 0: return launch_adj_ws<L, 0, FULL>(a, ms, s);
    case 1: return launch_adj_ws<L, 1, FULL>(a, ms, s);
    case 2: return launch_adj_ws<L, 2, FULL>(a, ms, s);
    case 3: return launch_adj_ws<L, 3, FULL>(a, ms, s);
    case 4: return launch_adj_ws<L, 4, FULL>(a, ms, s);
    default: return launch_adj_ws<L, 5, FULL>(a, ms, s);
  }
}

template <int L>
int run_zy_adj(const ZYArgs& a, cudaStream_t s) {
  if (a.nzout <= 0 || a.nout <= 0) return 0;
  const int c = single_component(a.need[0][0]);
  if (a.nin == 1 && a.nout == 1 && a.nzin == 1 && c >= 0) {
    if constexpr (yz_ws_plan<L>()) {
      CUtensorMap ms;
      if (a.Ts && a.nzin_total > 0 && a.n_src <= L / 2 &&
          slice_map(&ms, a.Ts, (long long)a.nzin_total * (L / 2 + 1), a.P, slice_box_rows<L>()))
        return a.n_out == L / 2 ? launch_adj_ws_c<L, true>(a, c, ms, s) : launch_adj_ws_c<L, false>(a, c, ms, s);
    }
    if (a.gsrc) return -1;  // the source's y transform is only done on the warp-specialized path
    return launch_adj<L, true>(a, c, s);
  }
  if (a.gsrc) return -1;
  return launch_adj<L, false>(a, -1, s);
}

template <int L>
constexpr bool ws_length() {
  return yz_ws_plan<L>();
}

template <int L>
size_t staged_smem() {
  return (size_t)(L + L * TB + 2 * (L / 2) * TB) * sizeof(float2) + (size_t)2 * (L / 2 + 1) * TB * sizeof(float);
}

template <int L>
int launch_fwd_staged(const YZArgs& a, int c, int nch, cudaStream_t s) {
  const size_t sm = staged_smem<L>();
  static bool init = false;
  if (!init) {
    if (cudaFuncSetAttribute(k_yz_fwd_staged<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) !=
        cudaSuccess)
      return -1;
    init = true;
  }
  k_yz_fwd_staged<L><<<dim3(a.P / TB, nch), NTF, sm, s>>>(a, c);
  return 0;
}

template <int L, bool SIMPLE>
int launch_fwd(const YZArgs& a, int c, int nch, cudaStream_t s) {
  const size_t sm = fused_smem<L>();
  static bool init = false;
  if (!init) {
    if (cudaFuncSetAttribute(k_yz_fwd<L, SIMPLE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) !=
        cudaSuccess)
      return -1;
    init = true;
  }
  k_yz_fwd<L, SIMPLE><<<dim3(a.P / TB, nch), NTF, sm, s>>>(a, c);
  return 0;
}

template <int L, int C, bool FULL>
int launch_fwd_ws(const YZArgs& a, const CUtensorMap& mslice, cudaStream_t s) {
  constexpr size_t sm = ws_smem<L>();
  static bool init = false;
  if (!init) {
    if (cudaFuncSetAttribute(k_yz_fwd_ws<L, C, FULL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) !=
        cudaSuccess)
      return -1;
    init = true;
  }
  const long long items = (long long)(a.P / TB) * a.nzin;
  const int blocks = (int)(items < sm_count() ? items : sm_count());  // one resident block per SM
  return launch_k(k_yz_fwd_ws<L, C, FULL>, dim3(blocks), dim3(NTF), sm, s, a.pdl != 0, a, mslice) == cudaSuccess
             ? 1  // 1: segment partials written; launch_yz_finish completes the target plane
             : -1;
}
template <int L, bool FULL>
int launch_fwd_ws_c(const YZArgs& a, int c, const CUtensorMap& ms, cudaStream_t s) {
  switch (c) {
    case 0: return launch_fwd_ws<L, 0, FULL>(a, ms, s);
    case 1: return launch_fwd_ws<L, 1, FULL>(a, ms, s);
    case 2: return launch_fwd_ws<L, 2, FULL>(a, ms, s);
    case 3: return launch_fwd_ws<L, 3, FULL>(a, ms, s);
    case 4: return launch_fwd_ws<L, 4, FULL>(a, ms, s);
    default: return launch_fwd_ws<L, 5, FULL>(a, ms, s);
  }
}

template <int L>
int launch_fwd_single(const YZArgs& a, int c, int nch, cudaStream_t s) {
  if constexpr (yz_ws_plan<L>()) {
    // needs the segment buffers, the scaled tensor component, and at most two column
    // blocks per block (blocks >= P / TB)
    CUtensorMap ms;
    if (a.n_in <= L / 2 && a.seg && a.yrows && a.Ts && a.P / TB <= sm_count() && sm_count() <= kFinishMaxBlocks &&
        slice_map(&ms, a.Ts, (long long)a.nz_total * (L / 2 + 1), a.P, slice_box_rows<L>()))
      return a.n_in == L / 2 ? launch_fwd_ws_c<L, true>(a, c, ms, s) : launch_fwd_ws_c<L, false>(a, c, ms, s);
  }
  return launch_fwd_staged<L>(a, c, nch, s);
}

template <int L>
int run_yz_fwd(const YZArgs& a, cudaStream_t s) {
  const int nch = (a.nzin + a.zchunk - 1) / a.zchunk;
  const int c = single_component(a.need[0]);
  const int r = a.nin == 1 && c >= 0 ? launch_fwd_single<L>(a, c, nch, s) : launch_fwd<L, false>(a, -1, nch, s);
  if (r != 0) return r;
  const long long plane = (long long)L * a.P;
  const long long b = (plane + 255) / 256;
  k_yz_reduce<<<(int)(b > 2048 ? 2048 : b), 256, 0, s>>>(reinterpret_cast<const float2*>(a.part), nch, plane,
                                                        a.out + a.out_slot * a.out_cstride + a.zout * plane);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace

int launch_zy_adj(int L, const ZYArgs& a, cudaStream_t s) {
  switch (L) {
#define TM_CASE(LL) \
  case LL:          \
    return run_zy_adj<LL>(a, s);
    TM_FOR_EACH_L(TM_CASE)
#undef TM_CASE
  }
  return -2;
}

template <int L>
int run_yz_finish(const YZArgs& a, cudaStream_t s) {
  if constexpr (yz_ws_plan<L>()) {
    const long long items = (long long)(a.P / TB) * a.nzin;
    const int blocks = (int)(items < sm_count() ? items : sm_count());  // the forward's grid
    return launch_k(k_yz_finish<L>, dim3(a.P / TB, TB / kFinishLines), dim3(kFinishThreads), 0, s, a.pdl != 0, a,
                    blocks) == cudaSuccess
               ? 0
               : -1;
  }
  return -1;
}

int launch_yz_finish(int L, const YZArgs& a, cudaStream_t s) {
  switch (L) {
#define TM_CASE(LL) \
  case LL:          \
    return run_yz_finish<LL>(a, s);
    TM_FOR_EACH_L(TM_CASE)
#undef TM_CASE
  }
  return -2;
}

bool zy_adj_ws_length(int L) {
  switch (L) {
#define TM_CASE(LL) \
  case LL:          \
    return ws_length<LL>();
    TM_FOR_EACH_L(TM_CASE)
#undef TM_CASE
  }
  return false;
}

int launch_yz_fwd(int L, const YZArgs& a, cudaStream_t s) {
  switch (L) {
#define TM_CASE(LL) \
  case LL:          \
    return run_yz_fwd<LL>(a, s);
    TM_FOR_EACH_L(TM_CASE)
#undef TM_CASE
  }
  return -2;
}

}  // namespace tmk
