// BF16 MLP layers on the tensor cores (tcgen05.mma, accumulator in TMEM,
// operands staged by 2-D TMA), and the 128-bit gather that turns the
// surviving fp32 tuple rows into the dense BF16 operand of the first layer.
//
// Y[m][n] = relu(sum_k X[m][k] W[n][k] + b[n]) for m < *count: CTA tiles of
// 128 rows x NT columns, K in 64-element (128-byte, 128B-swizzled) slices,
// persistent over tiles, warp-specialised like the conv kernel (TMA warp,
// MMA warp, four epilogue warps), two TMEM accumulators.  The UDF's last
// layer (one output) is folded into the epilogue of the last hidden layer:
// each row leaves one partial head . relu(...) per column tile, summed in a
// fixed order by a finalize kernel.
#include <string>

#include "common.cuh"
#include "tc_common.cuh"
#include "tc_gemm.h"

namespace hydro {

namespace {

using namespace tcx;
thread_local std::string g_gemm_err;

template <int NT, int S>
struct GemmCfg {
    static constexpr int A_BYTES = 128 * 128;   // 128 rows x 64 bf16
    static constexpr int B_BYTES = NT * 128;    // NT rows x 64 bf16
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int TMEM_COLS = 2 * NT;
    static constexpr int SMEM = S * STAGE + 1024 + 256;
};

template <int NT, int S>
__global__ void __launch_bounds__(192, 1)
k_gemm_bf16_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const int *count,
               int K, int N, const float *__restrict__ bias, __nv_bfloat16 *Y, const float *__restrict__ head_w,
               float *partials, unsigned int *err) {
    using C = GemmCfg<NT, S>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + S * C::STAGE);
    uint64_t *empty = full + S;
    uint64_t *tfull = empty + S;
    uint64_t *tempty = tfull + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tempty + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int M = *count;
    const int tiles_n = N / NT;
    const int total = ((M + 127) / 128) * tiles_n;
    const int kblocks = K / 64;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 4);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"((uint32_t)C::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0, issued = 0, last_par = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
                const int m0 = (t / tiles_n) * 128, n0 = (t % tiles_n) * NT;
                for (int kb = 0; kb < kblocks; ++kb) {
                    if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag)) {
                        ok = false;
                        break;
                    }
                    unsigned char *sa = smem + s * C::STAGE;
                    mbar_expect_tx(&full[s], (uint32_t)C::STAGE);
                    tma_load_2d(sa, &tmA, &full[s], kb * 64, m0);
                    tma_load_2d(sa + C::A_BYTES, &tmB, &full[s], kb * 64, n0);
                    issued |= 1u << s;
                    last_par = (last_par & ~(1u << s)) | (ph << s);
                    if (++s == S) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
            }
            if (!ok) {
                *abort_flag = 1;
                volatile int never = 0;
                for (int k = 0; k < S; ++k)
                    if (issued & (1u << k)) mbar_wait(&full[k], (last_par >> k) & 1u, &never, 100000000ull);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(128, NT);
            int s = 0;
            uint32_t ph = 0;
            int tl = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < total && ok; t += gridDim.x, ++tl) {
                const int buf = tl & 1;
                const uint32_t tph = (uint32_t)(tl >> 1) & 1u;
                if (!mbar_wait(&tempty[buf], tph ^ 1u, abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t dt = tmem_base + (uint32_t)(buf * NT);
                for (int kb = 0; kb < kblocks; ++kb) {
                    if (!mbar_wait(&full[s], ph, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(smem + s * C::STAGE);
                    const uint32_t sb = sa + C::A_BYTES;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        mma_bf16(dt, smem_desc(sa + kk * 32, 1024, 2u), smem_desc(sb + kk * 32, 1024, 2u), idesc,
                                 (kb | kk) != 0);
                    mma_commit(&empty[s]);
                    if (++s == S) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
                if (ok) mma_commit(&tfull[buf]);
            }
            if (!ok) *abort_flag = 1;
        }
    } else {
        const int qtr = warp & 3;
        const int row = qtr * 32 + lane;
        int tl = 0;
        for (int t = blockIdx.x; t < total; t += gridDim.x, ++tl) {
            const int buf = tl & 1;
            const uint32_t tph = (uint32_t)(tl >> 1) & 1u;
            if (!mbar_wait(&tfull[buf], tph, abort_flag)) {
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            const int tn = t % tiles_n;
            const int m = (t / tiles_n) * 128 + row, n0 = tn * NT;
            float hsum = 0.f;
#pragma unroll 1
            for (int c0 = 0; c0 < NT; c0 += 32) {
                uint32_t r[32];
                tmem_ld32(tmem_base + ((uint32_t)(qtr * 32) << 16) + (uint32_t)(buf * NT + c0), r);
                tmem_ld_wait();
                if (head_w) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        float v = __uint_as_float(r[j]) + __ldg(bias + n0 + c0 + j);
                        v = v > 0.f ? v : 0.f;
                        hsum = fmaf(__ldg(head_w + n0 + c0 + j), v, hsum);
                    }
                } else if (m < M) {
                    uint32_t pk[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        float v0 = __uint_as_float(r[2 * j]) + __ldg(bias + n0 + c0 + 2 * j);
                        float v1 = __uint_as_float(r[2 * j + 1]) + __ldg(bias + n0 + c0 + 2 * j + 1);
                        v0 = v0 > 0.f ? v0 : 0.f;
                        v1 = v1 > 0.f ? v1 : 0.f;
                        pk[j] = pack_bf16x2(v0, v1);
                    }
                    uint4 *dst = reinterpret_cast<uint4 *>(Y + (size_t)m * N + n0 + c0);
#pragma unroll
                    for (int j = 0; j < 4; ++j) dst[j] = make_uint4(pk[4 * j], pk[4 * j + 1], pk[4 * j + 2], pk[4 * j + 3]);
                }
            }
            if (head_w && m < M) partials[(size_t)m * tiles_n + tn] = hsum;
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[buf]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                     "r"((uint32_t)C::TMEM_COLS)
                     : "memory");
    }
    if (threadIdx.x == 0 && *abort_flag) atomicOr(err, ERR_TC_TIMEOUT);
}

// Gather the listed fp32 rows into a dense BF16 matrix, 8 values per thread:
// two 128-bit loads, one 128-bit store.
__global__ void k_gather_bf16(const int *count, const int *rows, const float *X, int ldx, int K,
                              __nv_bfloat16 *out) {
    const int M = *count;
    const int per_row = K / 8;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)M * per_row;
         i += (long long)gridDim.x * blockDim.x) {
        const int m = (int)(i / per_row), q = (int)(i % per_row);
        const float4 *src = reinterpret_cast<const float4 *>(X + (size_t)(rows ? rows[m] : m) * ldx) + 2 * q;
        const float4 a = src[0], b = src[1];
        const uint4 v = make_uint4(pack_bf16x2(a.x, a.y), pack_bf16x2(a.z, a.w), pack_bf16x2(b.x, b.y),
                                   pack_bf16x2(b.z, b.w));
        reinterpret_cast<uint4 *>(out + (size_t)m * K)[q] = v;
    }
}

using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                              const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

template <int NT, int S>
cudaError_t gemm_smem() {
    return cudaFuncSetAttribute(k_gemm_bf16_tc<NT, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                GemmCfg<NT, S>::SMEM);
}

constexpr int kS256 = 4, kS128 = 6, kS64 = 8;

bool encode2d(EncodeFn enc, CUtensorMap *m, const void *base, int inner, long long outer, int box_inner,
              int box_outer) {
    const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    const cuuint64_t strides[1] = {(cuuint64_t)inner * 2};
    const cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer};
    const cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool tc_gemm_supported(int K, int N) { return K >= 64 && K % 64 == 0 && N >= 64 && N % 64 == 0 && K <= 65536; }

hydro_status tc_gemm_init(void **encode) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult qr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr);
    if (e != cudaSuccess || qr != cudaDriverEntryPointSuccess || !fn) {
        g_gemm_err = "cuTensorMapEncodeTiled entry point not available";
        return HYDRO_ECUDA;
    }
    *encode = fn;
    cudaError_t r = gemm_smem<256, kS256>();
    if (r == cudaSuccess) r = gemm_smem<128, kS128>();
    if (r == cudaSuccess) r = gemm_smem<64, kS64>();
    if (r != cudaSuccess) {
        g_gemm_err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(r);
        return HYDRO_ECUDA;
    }
    return HYDRO_OK;
}

hydro_status tc_gemm_run(void *encode, const int *count, const __nv_bfloat16 *X, int K, const __nv_bfloat16 *W,
                         const float *bias, int N, __nv_bfloat16 *Y, int max_rows, int sms, cudaStream_t st,
                         unsigned int *err, const float *head_w, float *partials) {
    if (!encode || !tc_gemm_supported(K, N) || max_rows < 1) {
        g_gemm_err = "tensor-core GEMM not ready or shape unsupported";
        return HYDRO_EUNSUPPORTED;
    }
    EncodeFn enc = reinterpret_cast<EncodeFn>(encode);
    const int NT = N % 256 == 0 ? 256 : N % 128 == 0 ? 128 : 64;
    CUtensorMap tmA, tmB;
    if (!encode2d(enc, &tmA, X, K, max_rows, 64, 128) || !encode2d(enc, &tmB, W, K, N, 64, NT)) {
        g_gemm_err = "cuTensorMapEncodeTiled failed";
        return HYDRO_ECUDA;
    }
    const long long tiles = (long long)((max_rows + 127) / 128) * (N / NT);
    const int grid = (int)(tiles < sms ? tiles : sms);
    if (NT == 256)
        k_gemm_bf16_tc<256, kS256><<<grid, 192, GemmCfg<256, kS256>::SMEM, st>>>(tmA, tmB, count, K, N, bias, Y,
                                                                                 head_w, partials, err);
    else if (NT == 128)
        k_gemm_bf16_tc<128, kS128><<<grid, 192, GemmCfg<128, kS128>::SMEM, st>>>(tmA, tmB, count, K, N, bias, Y,
                                                                                 head_w, partials, err);
    else
        k_gemm_bf16_tc<64, kS64><<<grid, 192, GemmCfg<64, kS64>::SMEM, st>>>(tmA, tmB, count, K, N, bias, Y, head_w,
                                                                             partials, err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        g_gemm_err = std::string("launch: ") + cudaGetErrorString(e);
        return HYDRO_ECUDA;
    }
    return HYDRO_OK;
}

int tc_gemm_col_tiles(int N) { return N / (N % 256 == 0 ? 256 : N % 128 == 0 ? 128 : 64); }

void launch_gather_bf16(const int *count, const int *rows, const float *X, int ldx, int K, __nv_bfloat16 *out,
                        int max_rows, int sms, cudaStream_t st) {
    long long work = (long long)max_rows * (K / 8);
    int grid = (int)((work + 255) / 256);
    if (grid > sms * 8) grid = sms * 8;
    if (grid < 1) grid = 1;
    k_gather_bf16<<<grid, 256, 0, st>>>(count, rows, X, ldx, K, out);
}

const char *tc_gemm_last_error() { return g_gemm_err.c_str(); }

}  // namespace hydro
