/*
 * rihv_nn.h - C ABI of the warm-start network's layer operations (part of
 * librihv.so).
 *
 * The network is not in the paper: it is this project's learned warm start
 * for the FISTA reconstruction (a small 3D U-Net that maps the back-propagated
 * hologram H^H b to an initial volume). Its layers run in these kernels:
 * BF16 activations and weights, 3x3x3 convolutions on 5th-generation tensor
 * cores (tcgen05) with FP32 accumulation in tensor memory.
 *
 * Conventions
 *  - One sample, channels last: a tensor with C channels over a d x h x w
 *    volume is [voxel][C], voxel = (z*h + y)*w + x. BF16 tensors are passed as
 *    uint16_t bit patterns (device memory, 16-byte aligned).
 *  - Channel counts of convolutions are multiples of 16 (pad with zero
 *    channels); c_out <= 256.
 *  - Weights W[c_out][27][c_in], tap = (dz+1)*9 + (dy+1)*3 + (dx+1), zero
 *    padding of one voxel.
 *  - All calls queue work on `stream` (cudaStream_t or NULL) and return.
 *    Errors: RIHV_ERR_INVALID_ARG for bad sizes or pointers (checked first),
 *    RIHV_ERR_CUDA for launch failures. `err_flag` (device int, may be NULL
 *    where noted) is set to 1 if a kernel's bounded wait gave up.
 */
#ifndef RIHV_NN_H
#define RIHV_NN_H

#include <stddef.h>
#include <stdint.h>

#include "rihv.h"

#ifdef __cplusplus
extern "C" {
#endif

/* y = relu?(conv3d(x, W) + bias). x: BF16 [v][c_in]; bias: FP32 [c_out] or
 * NULL; y: BF16 [v][c_out] (out_f32 = 0) or FP32 [v][c_out] (out_f32 = 1). */
rihv_status rihv_nn_conv3d(const uint16_t* x, const uint16_t* w, const float* bias, void* y,
                           int d, int h, int wd, int c_in, int c_out, int relu, int out_f32,
                           int* err_flag, void* stream);

/* Input gradient gx = conv3d^T(gy, W): gy BF16 [v][c_out]; gx BF16 [v][c_in]
 * (out_f32 = 0) or FP32 (out_f32 = 1). */
rihv_status rihv_nn_conv3d_dgrad(const uint16_t* gy, const uint16_t* w, void* gx, int d, int h,
                                 int wd, int c_in, int c_out, int out_f32, int* err_flag,
                                 void* stream);

/* Bytes of workspace rihv_nn_conv3d_wgrad needs for this shape. */
size_t rihv_nn_conv3d_wgrad_workspace(int d, int h, int wd, int c_in, int c_out);

/* Weight gradient gw[o][t][c] = sum_v gy[v][o] x[v + off_t][c] (FP32 output,
 * overwritten). workspace: device memory of at least the size above. */
rihv_status rihv_nn_conv3d_wgrad(const uint16_t* x, const uint16_t* gy, float* gw, int d, int h,
                                 int wd, int c_in, int c_out, void* workspace,
                                 size_t workspace_bytes, int* err_flag, void* stream);

/* gb[c] = sum_v gy[v][c] (FP32, overwritten; FP64 partial sums in fixed
 * order). work: device memory of at least 256 * c * 8 bytes. */
rihv_status rihv_nn_bias_grad(const uint16_t* gy, float* gb, size_t voxels, int c, void* work,
                              void* stream);

/* out = (y > 0) ? g : 0, elementwise over n BF16 values (ReLU backward from
 * the layer's output y). */
rihv_status rihv_nn_relu_grad(const uint16_t* g, const uint16_t* y, uint16_t* out, size_t n,
                              void* stream);

/* 2x2x2 mean pooling of x [d][h][wd][c] (even sizes) into y, and its adjoint
 * (gx receives gy/8 in each cell). */
rihv_status rihv_nn_avgpool2(const uint16_t* x, uint16_t* y, int d, int h, int wd, int c,
                             void* stream);
rihv_status rihv_nn_avgpool2_grad(const uint16_t* gy, uint16_t* gx, int d, int h, int wd, int c,
                                  void* stream);

/* Nearest-neighbour 2x upsampling of x [d][h][wd][c] into y [2d][2h][2wd][c],
 * and its adjoint (gx sums gy over each 2x2x2 cell). */
rihv_status rihv_nn_upsample2(const uint16_t* x, uint16_t* y, int d, int h, int wd, int c,
                              void* stream);
rihv_status rihv_nn_upsample2_grad(const uint16_t* gy, uint16_t* gx, int d, int h, int wd, int c,
                                   void* stream);

/* out = a + b over n BF16 values (gradient accumulation at skip connections). */
rihv_status rihv_nn_add(const uint16_t* a, const uint16_t* b, uint16_t* out, size_t n,
                        void* stream);

/* Channel concatenation out[v] = (a[v], b[v]) and its adjoint (split). */
rihv_status rihv_nn_concat(const uint16_t* a, const uint16_t* b, uint16_t* out, size_t voxels,
                           int ca, int cb, void* stream);
rihv_status rihv_nn_split(const uint16_t* g, uint16_t* ga, uint16_t* gb, size_t voxels, int ca,
                          int cb, void* stream);

/* Network input from a complex64 volume: channel 0 = scale * Re, channel 1 =
 * scale * Im, channels 2..c-1 = 0 (BF16 [v][c]). */
rihv_status rihv_nn_pack_input(const void* vol_c64, uint16_t* out, size_t voxels, int c,
                               float scale, void* stream);

/* Complex64 volume from the network output: vol = scale * (y0 + i y1)
 * + base_scale * base, where y is FP32 [v][c] and base an optional complex64
 * volume (NULL: no base term). vol may alias base. */
rihv_status rihv_nn_unpack_output(const float* y, const void* base_c64, float base_scale,
                                  void* vol_c64, size_t voxels, int c, float scale, void* stream);

/* Mean squared error between the output (channels 0 and 1 of FP32 y [v][c])
 * and target/scale (complex64 volume): loss = mean over voxels of
 * |y0 + i y1 - target/scale|^2 written to *loss (device double, FP64
 * accumulation); gy (BF16 [v][c]) receives its gradient, 0 in channels >= 2.
 * work: device memory of at least 8 * 1024 bytes. */
rihv_status rihv_nn_mse_grad(const float* y, const void* target_c64, uint16_t* gy, double* loss,
                             size_t voxels, int c, float scale, void* work, void* stream);

/* One Adam step (Kingma and Ba) on n FP32 parameters with FP32 gradient and
 * moments; writes the BF16 copy the convolutions read. step >= 1. */
rihv_status rihv_nn_adam(float* param, const float* grad, float* m, float* v, uint16_t* param_bf16,
                         size_t n, float lr, float beta1, float beta2, float eps, int step,
                         void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RIHV_NN_H */
