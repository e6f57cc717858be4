// Small helper kernels for the synchronous score API.
#include "common.cuh"
#include "internal.h"

namespace hydro {

__global__ void k_f32_to_f64(const float *src, double *dst, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = (double)src[i];
}

// list[i] = start + i for i < n, *count = n.
__global__ void k_identity_list(int *list, int *count, int start, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) list[i] = start + i;
    if (blockIdx.x == 0 && threadIdx.x == 0) *count = n;
}

void launch_f32_to_f64(const float *src, double *dst, int n, cudaStream_t st) {
    const int g = n > 0 ? (n + 255) / 256 : 1;
    k_f32_to_f64<<<g, 256, 0, st>>>(src, dst, n);
}

void launch_identity_list(int *list, int *count, int start, int n, cudaStream_t st) {
    const int g = n > 0 ? (n + 255) / 256 : 1;
    k_identity_list<<<g, 256, 0, st>>>(list, count, start, n);
}

}  // namespace hydro
