// Tensor-core (tcgen05, TMA-fed) BF16 conv3x3 layer for the CNN UDFs.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <vector>

#include "../../include/hydro.h"

namespace hydro {

struct TcConvPlan {
    bool ready = false;
    int device = -1;
    void *encode = nullptr;   // cuTensorMapEncodeTiled entry point
    int smem_per_sm = 0;      // shared memory per SM (bytes)
};

// Whether a layer of this shape runs on the tensor-core kernel.
bool tc_conv_supported(int cin, int cout, int H, int W);
// First conv layer on the tensor cores (BF16 output): uint8 frames with C0 <= 3
// channels, Cout == 32, 8 <= W <= 512, H*W a multiple of 128 below 2^22,
// batches of max_frames * H * W < 2^31 pixels, and fp32 weights
// w [32][C0][3][3] and biases b [32] (host) of moderate size.
bool tc_conv1_supported(int C0, int H, int W, int Cout, int max_frames, const float *w, const float *b);
hydro_status launch_conv1_tc(TcConvPlan *plan, const int *count, const int *list, const unsigned char *frames,
                             int C0, int H, int Wd, const void *Bt, __nv_bfloat16 *out, int max_frames, int sms,
                             unsigned int *err, cudaStream_t st);
// The first layer's FP16 weight tile with the bias folded in (device copy
// passed to launch_conv1_tc as Bt): w [32][C0][3][3], b [32].
void tc_conv1_pack_weights(const float *w, const float *b, int C0, std::vector<__half> &out);
// Repack fp32 weights [cout][cin][3][3] into the kernel's bf16 layout.
void tc_conv_pack_weights(const float *w, int cin, int cout, std::vector<__nv_bfloat16> &out);
// FP32-accurate split form: [plane(hi, lo)][chunk of 32][kx][ky][cout][32] fp32.
void tc_conv_pack_weights_split(const float *w, int cin, int cout, std::vector<float> &out);
// Split-BF16 form: [plane(bf16(w), bf16(w - plane 0))][chunk][kx][ky][cout][chunk] bf16.
void tc_conv_pack_weights_split_bf16(const float *w, int cin, int cout, std::vector<__nv_bfloat16> &out);
hydro_status tc_conv_init(TcConvPlan *plan, int device);
// out[m] = relu(conv3x3(in[m]) + bias) for m < *count (device), NHWC bf16.
// With head_w != nullptr the layer is the UDF's last: nothing is stored to
// `out`; instead the frame's tc_conv_head_parts(...) partials (from
// partials + m * that count on) receive sums over 32 pixels of
// head_w . relu(conv + bias) (4 partials per 128-pixel subtile).
hydro_status tc_conv_run(TcConvPlan *plan, const int *count, const void *in, int cin, int H, int W,
                         const void *wpacked, const float *bias, int cout, void *out, int max_frames, int sms,
                         cudaStream_t st, unsigned int *err, const float *head_w = nullptr,
                         float *partials = nullptr, int mode = 0);
// mode 1: 3xTF32 (FP32-accurate up to the accumulation): `in` and `out` are
// fp32 [frame][pixel][hi(C) | lo(C)] TF32 planes and wpacked comes from
// tc_conv_pack_weights_split.  mode 2: split BF16, `in` and `out` bf16
// [frame][pixel][hi(C) | lo(C)] and wpacked from tc_conv_pack_weights_split_bf16.
// Head partials per frame that a fused-head layer leaves (the window kernel of
// the BF16 64-output layers has 3 subtiles of 128 padded pixels per tile),
// and the most any layer of an H x W frame leaves (for sizing the buffer).
int tc_conv_head_parts(int cin, int cout, int H, int W, int mode);
int tc_conv_max_head_parts(int H, int W);
// score[m] = hb + sum(partials of frame m) / HW for m < *count.
void tc_head_finalize(const int *count, const float *partials, int parts_per_frame, double hb, int HW,
                      float *score, int max_frames, int sms, cudaStream_t st);
void tc_conv_destroy(TcConvPlan *plan);
// Launch the bounded-wait self-test (an mbarrier wait nothing completes).
cudaError_t wait_selftest(unsigned long long limit_ns, int *d_status, cudaStream_t st);
const char *tc_conv_last_error();

}  // namespace hydro
