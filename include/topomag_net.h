/*
 * topomag_net -- kernels of the learned warm start (a small 3-D U-Net that maps
 * a target specification to an initial density). The paper has no counterpart:
 * its optimizer starts from rho = 1 (Sec. "Validation and Benchmarks"); here the
 * optimizer always refines the network's output, so the network can only
 * change the number of optimizer steps, never the answer.
 *
 * Conventions: device pointers on the current device, caller-owned; `stream`
 * is a cudaStream_t. Activations are channels-last [N][D][H][W][C] bfloat16
 * with C a multiple of 16; activation gradients are float32 in the same
 * layout. Weights: float32 master [27][Cin][Cout] with tap =
 * (dz+1)*9 + (dy+1)*3 + (dx+1); bfloat16 copies Wf (forward) and Wb (backward
 * data), each 27*Cin*Cout values packed by tmn_pack_conv_weights in the operand
 * layout of the tensor-core kernels (opaque to callers: make them with
 * tmn_pack_conv_weights or tmn_adamw). Convolutions are 3x3x3, stride 1, zero
 * padding 1. Return 0, or -1 (bad argument), -4 (CUDA error), -5 (work buffer
 * too small).
 */
#ifndef TOPOMAG_NET_H
#define TOPOMAG_NET_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* out = relu?(conv(in, W) + bias), bfloat16; Cin % 16 == 0, Cout in {16, 32, 64}. An implicit
 * GEMM on the fifth-generation tensor cores: M = 128 voxels, N = Cout, the float32
 * accumulator in tensor memory, bfloat16 operands. For W in {8, 16, 32, 64} (and `in` 16-byte
 * aligned) a block stages its halo rows once and every tap reads them; other grids gather
 * each voxel's shifted channels per tap. Same products and float32 sums either way. */
int tmn_conv3d_forward(const void* in, const void* Wf, const float* bias, void* out, int N, int D, int H, int W,
                       int Cin, int Cout, int relu, void* stream);

/* din (+)= conv^T(dout, W), float32; Cout % 16 == 0, Cin in {16, 32, 48, 64, 96}. dout is
 * rounded to bfloat16 as a product operand; the same tensor-core kernels as the forward
 * (halo tiles for W in {8, 16, 32, 64}), N = Cin. accumulate: add to din instead of
 * overwriting it. */
int tmn_conv3d_backward_data(const float* dout, const void* Wb, float* din, int N, int D, int H, int W, int Cin,
                             int Cout, int accumulate, void* stream);

/* dW[27][Cin][Cout] and db[Cout] (overwritten) from in (bfloat16) and dout (float32, rounded
 * to bfloat16 where it is a product operand, as for the data gradient; float32 for db). An
 * implicit GEMM on the fifth-generation tensor cores with rows (tap, ci), columns co and the
 * voxels as the reduction; float32 partial sums per block of voxels, added in a fixed order.
 * Cin % 16 == 0, Cout in {16, 32, 64}. work: float32 scratch of work_floats >=
 * tmn_conv3d_backward_weight_work(N*D*H*W, Cin, Cout) elements (it holds the bfloat16 copy
 * of dout and the partials; more allows more blocks); -5 if smaller. */
int tmn_conv3d_backward_weight(const void* in, const float* dout, float* dW, float* db, float* work,
                               long long work_floats, int N, int D, int H, int W, int Cin, int Cout, void* stream);
long long tmn_conv3d_backward_weight_work(long long nvox, int Cin, int Cout);

/* Error word of the tensor-core kernels since the last call (bit 0: a bounded wait for a
 * copy or an MMA ran out, the results of that launch are invalid), then cleared.
 * Synchronous. */
int tmn_status(unsigned* out);

/* g[i] = 0 where act[i] <= 0 (ReLU backward through the stored activation). */
int tmn_relu_backward(float* g, const void* act, long long n, void* stream);

/* 2x2x2 average pooling of [N][D][H][W][C] into [N][D/2][H/2][W/2][C], and its adjoint. */
int tmn_pool(const void* in, void* out, int N, int D, int H, int W, int C, void* stream);
int tmn_pool_backward(const float* gout, float* gin, int N, int D, int H, int W, int C, int accumulate, void* stream);

/* out[.., 0:C1] = nearest 2x upsampling of x [N][D/2][H/2][W/2][C1], out[.., C1:C1+C2] = skip;
 * backward: gx (coarse grid) and gskip, both overwritten. D, H, W are the fine sizes. */
int tmn_upcat(const void* x, const void* skip, void* out, int N, int D, int H, int W, int C1, int C2, void* stream);
int tmn_upcat_backward(const float* gout, float* gx, float* gskip, int N, int D, int H, int W, int C1, int C2,
                       void* stream);

/* rho0 = sigmoid(sum_c w[c] x[c] + b) per voxel; backward of the mean squared error against
 * target: gx (overwritten), out[0:C] = dL/dw, out[C] = dL/db, out[C+1] = loss; work >= 256*(C+2). */
int tmn_head_forward(const void* x, const float* w, const float* b, float* rho, long long nvox, int C, void* stream);
int tmn_head_backward(const void* x, const float* w, const float* rho, const float* target, long long nvox, int C,
                      float* gx, float* work, float* out, void* stream);

/* AdamW step on float32 master weights (bias-corrected, step >= 1); if wf/wb are not NULL the
 * weights are a conv [27][cin][cout] and their bfloat16 Wf / Wb copies are refreshed. */
int tmn_adamw(float* w, const float* g, float* m, float* v, long long n, float lr, float b1, float b2, float eps,
              float wd, int step, void* wf, void* wb, int cin, int cout, void* stream);

/* Wf and Wb (bfloat16) from float32 master weights w [27][cin][cout]. */
int tmn_pack_conv_weights(const float* w, void* wf, void* wb, int cin, int cout, void* stream);

/* Network input from a target specification: channel 0 = mask footprint foot[N][H][W],
 * channel 1 = footprint * ht[n] (Ht_z / Ms), channel 2 = hgt[n] (plane height / 8), constant
 * along z; other channels zero. */
int tmn_spec_input(const uint8_t* foot, const float* ht, const float* hgt, void* out, int N, int D, int H, int W,
                   int C, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TOPOMAG_NET_H */
