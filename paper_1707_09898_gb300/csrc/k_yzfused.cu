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
#include "fft.cuh"
#include "internal.h"

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

template <int L>
int run_zy_adj(const ZYArgs& a, cudaStream_t s) {
  if (a.nzout <= 0 || a.nout <= 0) return 0;
  const int c = single_component(a.need[0][0]);
  if (a.nin == 1 && a.nout == 1 && a.nzin == 1 && c >= 0) return launch_adj<L, true>(a, c, s);
  return launch_adj<L, false>(a, -1, s);
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

template <int L>
int run_yz_fwd(const YZArgs& a, cudaStream_t s) {
  const int nch = (a.nzin + a.zchunk - 1) / a.zchunk;
  const int c = single_component(a.need[0]);
  if ((a.nin == 1 && c >= 0 ? launch_fwd_staged<L>(a, c, nch, s) : launch_fwd<L, false>(a, -1, nch, s)) != 0)
    return -1;
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
