// y and z passes of the stray-field convolution (Sec. "Discretization", Eq. (convolution)).
//
// y pass: tiles of 16 contiguous kx columns; forward transforms read y < n_in
// (the rest of the length-L line is the zero padding) and write all L
// digit-reversed positions; inverse transforms read all positions and keep the
// first n_out rows (the crop).
// z pass: the forward z transform of the three magnetization components, the
// product with the symmetric 3x3 tensor N^(k) (real after the transform, stored
// once for kx, ky, kz in [0, L/2] and unfolded by parity), and the inverse z
// transform, fused per column so the spectrum of M never leaves shared memory.
#include "fft.cuh"
#include "internal.h"

namespace tmk {

namespace {

template <int L, bool INV>
__global__ void __launch_bounds__(kNT, 3) k_ypass(YArgs a) {
  constexpr int S = plan_stages(L);
  extern __shared__ __align__(16) unsigned char smem[];
  cx<float>* tw = reinterpret_cast<cx<float>*>(smem);
  cx<float>* tile = tw + L;
  load_twiddles<float, kNT>(tw, reinterpret_cast<const cx<float>*>(a.tw), L);
  const int chunk = blockIdx.x, z = blockIdx.y, c = blockIdx.z;
  const cx<float>* in =
      reinterpret_cast<const cx<float>*>(a.in) + c * a.in_cstride + z * a.in_zstride + chunk * TB;
  cx<float>* out = reinterpret_cast<cx<float>*>(a.out) + c * a.out_cstride + z * a.out_zstride + chunk * TB;
  __syncthreads();
  if (!INV) {
    dif_stage0_load<float, L, kNT>(tile, tw, [&](int pos, int line) {
      return pos < a.n_in ? in[pos * a.in_pstride + line] : zero<float>();
    });
    __syncthreads();
    DifRange<float, L, kNT, 1, S - 1>::run(tile, tw);
    dif_last_store<float, L, kNT>(tile, [&](int pos, int line, cx<float> v) { out[pos * a.out_pstride + line] = v; });
  } else {
    dit_last_load<float, L, kNT>(tile, [&](int pos, int line) { return in[pos * a.in_pstride + line]; });
    __syncthreads();
    DitRange<float, L, kNT, 1, S - 1>::run(tile, tw);
    dit_stage0_store<float, L, kNT>(tile, tw, [&](int pos, int line, cx<float> v) {
      if (pos < a.n_out) out[pos * a.out_pstride + line] = v;
    });
  }
}

// forward stages [s, e) on the three component tiles, one barrier per stage
template <int L, int s, int e>
__device__ __forceinline__ void dif3(cx<float>* t0, const cx<float>* tw) {
  if constexpr (s < e) {
#pragma unroll
    for (int c = 0; c < 3; c++) dif_stage<float, L, s, kNT>(t0 + c * L * TB, tw);
    __syncthreads();
    dif3<L, s + 1, e>(t0, tw);
  }
}
// inverse stages hi-1 down to lo
template <int L, int lo, int hi>
__device__ __forceinline__ void dit3(cx<float>* t0, const cx<float>* tw) {
  if constexpr (hi > lo) {
#pragma unroll
    for (int c = 0; c < 3; c++) dit_stage<float, L, hi - 1, kNT>(t0 + c * L * TB, tw);
    __syncthreads();
    dit3<L, lo, hi - 1>(t0, tw);
  }
}

template <int L>
__global__ void __launch_bounds__(kNT, 1) k_zpass(ZArgs a) {
  constexpr int S = plan_stages(L);
  constexpr int LH = L / 2;
  extern __shared__ __align__(16) unsigned char smem[];
  cx<float>* tw = reinterpret_cast<cx<float>*>(smem);
  cx<float>* tiles = tw + L;  // [3][L * TB]
  load_twiddles<float, kNT>(tw, reinterpret_cast<const cx<float>*>(a.tw), L);
  const int chunk = blockIdx.x;
  const int2 col = a.zcol[blockIdx.y];  // (ky position, ky)
  const int kyf = col.y <= a.Ly / 2 ? col.y : a.Ly - col.y;
  const float sy = col.y <= a.Ly / 2 ? 1.0f : -1.0f;
  cx<float>* base = reinterpret_cast<cx<float>*>(a.buf) + (long long)col.x * a.P + chunk * TB;
  __syncthreads();

#pragma unroll
  for (int c = 0; c < 3; c++) {
    const cx<float>* bc = base + c * a.cstride;
    dif_stage0_load<float, L, kNT>(tiles + c * L * TB, tw, [&](int pos, int line) {
      return pos < a.n_in ? bc[pos * a.zstride + line] : zero<float>();
    });
  }
  __syncthreads();
  dif3<L, 1, S - 1>(tiles, tw);

  // last forward stage, tensor product, first inverse stage (M = 1: R consecutive positions)
  {
    using SS = StageShape<L, S - 1>;
    constexpr int R = SS::R;
    constexpr int ITER = (SS::NU + kNT - 1) / kNT;
    const float* T = a.T + kyf * (long long)a.P + chunk * TB;
#pragma unroll 1
    for (int it = 0; it < ITER; it++) {
      const int u = it * kNT + threadIdx.x;
      if (SS::NU % kNT == 0 || u < SS::NU) {
        const int line = u % TB, g = u / TB;
        cx<float> v[3][R];
#pragma unroll
        for (int c = 0; c < 3; c++) {
#pragma unroll
          for (int q = 0; q < R; q++) v[c][q] = tiles[c * L * TB + (g * R + q) * TB + line];
          Dft<float, R, false>::run(v[c]);
        }
#pragma unroll
        for (int q = 0; q < R; q++) {
          const int kz = k_of_pos<L>(g * R + q);
          const int kzf = kz <= LH ? kz : L - kz;
          const float sz = kz <= LH ? 1.0f : -1.0f;
          const float* Tq = T + kzf * a.Tz + line;
          const float nxx = Tq[0], nyy = Tq[a.Tc], nzz = Tq[2 * a.Tc];
          const float nxy = sy * Tq[3 * a.Tc], nxz = sz * Tq[4 * a.Tc], nyz = sy * sz * Tq[5 * a.Tc];
          const cx<float> mx = v[0][q], my = v[1][q], mz = v[2][q];
          v[0][q] = mk(nxx * mx.x + nxy * my.x + nxz * mz.x, nxx * mx.y + nxy * my.y + nxz * mz.y);
          v[1][q] = mk(nxy * mx.x + nyy * my.x + nyz * mz.x, nxy * mx.y + nyy * my.y + nyz * mz.y);
          v[2][q] = mk(nxz * mx.x + nyz * my.x + nzz * mz.x, nxz * mx.y + nyz * my.y + nzz * mz.y);
        }
#pragma unroll
        for (int c = 0; c < 3; c++) {
          Dft<float, R, true>::run(v[c]);
#pragma unroll
          for (int q = 0; q < R; q++) tiles[c * L * TB + (g * R + q) * TB + line] = v[c][q];
        }
      }
    }
  }
  __syncthreads();
  dit3<L, 1, S - 1>(tiles, tw);
#pragma unroll
  for (int c = 0; c < 3; c++) {
    cx<float>* bc = base + c * a.cstride;
    dit_stage0_store<float, L, kNT>(tiles + c * L * TB, tw, [&](int pos, int line, cx<float> v) {
      if (pos < a.n_out) bc[pos * a.zstride + line] = v;
    });
  }
}

template <int L>
size_t ypass_smem() {
  return (size_t)(L + L * TB) * sizeof(float2);
}
template <int L>
size_t zsmem() {
  return (size_t)(L + 3 * L * TB) * sizeof(float2);
}

template <int L, bool INV>
int run_y(const YArgs& a, cudaStream_t s) {
  const size_t sm = ypass_smem<L>();
  static bool init = false;
  if (!init) {
    if (cudaFuncSetAttribute(k_ypass<L, INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
      return -1;
    init = true;
  }
  if (a.nplanes == 0) return 0;
  dim3 grid(a.P / TB, a.nplanes, 3);
  k_ypass<L, INV><<<grid, kNT, sm, s>>>(a);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

template <int L>
int run_z(const ZArgs& a, cudaStream_t s) {
  const size_t sm = zsmem<L>();
  static bool init = false;
  if (!init) {
    if (cudaFuncSetAttribute(k_zpass<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
      return -1;
    init = true;
  }
  dim3 grid(a.P / TB, a.Ly);
  k_zpass<L><<<grid, kNT, sm, s>>>(a);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace

size_t zpass_smem(int L) { return (size_t)(L + 3 * L * TB) * sizeof(float2); }

int launch_yfwd(int L, const YArgs& a, cudaStream_t s) {
  switch (L) {
#define TM_CASE(LL) \
  case LL:          \
    return run_y<LL, false>(a, s);
    TM_FOR_EACH_L(TM_CASE)
#undef TM_CASE
  }
  return -2;
}
int launch_yinv(int L, const YArgs& a, cudaStream_t s) {
  switch (L) {
#define TM_CASE(LL) \
  case LL:          \
    return run_y<LL, true>(a, s);
    TM_FOR_EACH_L(TM_CASE)
#undef TM_CASE
  }
  return -2;
}
int launch_zpass(int L, const ZArgs& a, cudaStream_t s) {
  switch (L) {
#define TM_CASE(LL) \
  case LL:          \
    return run_z<LL>(a, s);
    TM_FOR_EACH_L(TM_CASE)
#undef TM_CASE
  }
  return -2;
}

}  // namespace tmk
