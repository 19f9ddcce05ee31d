// Split-BF16 B-point DFT on the tensor cores (step a2 with sfft_opts.precision
// = 1): every (signal, loop) row of bucket sums z (B complex) times the real
// 2B x 2B DFT matrix, as one tcgen05 GEMM per launch group.
//
// With z and zhat interleaved (re, im), zhat = z W where, for theta =
// 2 pi j k / B (Eq. 2 with omega_B = exp(-2 pi i / B)),
//   W[2j][2k] = cos, W[2j][2k+1] = -sin, W[2j+1][2k] = sin, W[2j+1][2k+1] = cos.
// z and W are split into BF16 hi + lo parts (hi = bf16(v), lo = bf16(v - hi));
// zhat ~ z_hi W_hi + z_lo W_hi + z_hi W_lo, each product accumulated in FP32
// (the dropped z_lo W_lo is ~2^-16 of the result).  The three products run as
// three slices of the grid into three FP32 partial planes; the FFT/select
// kernel sums them in a fixed order, so the result is deterministic.
//
// GEMM kernel: a CTA computes a 128 x 128 tile of one product.  One thread
// issues TMA loads (cp.async.bulk.tensor, 128-byte swizzle) of 128 x 64 BF16
// tiles of A and of W^T into a 4-stage shared-memory ring and tcgen05.mma
// (kind::f16, BF16 in, FP32 accumulator in tensor memory, M = 128, N = 128,
// K = 16 per instruction); tcgen05.commit releases a stage when the MMAs that
// read it complete.  All four warps then read the accumulator back with
// tcgen05.ld (32 lanes x 32 columns at a time) and store it.  Every wait is
// bounded: on expiry the kernel records an error word, skips its stores and
// still frees its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>
#include <vector>

#include "device_common.cuh"
#include "sfft_internal.cuh"

namespace sfft {

namespace {

constexpr uint32_t kBM = 128, kBN = 128, kBK = 64, kStages = 4;
constexpr uint32_t kTileBytes = kBM * kBK * 2;  // one 128 x 64 BF16 tile (A or W^T): 16 KB
constexpr uint32_t kStageBytes = 2 * kTileBytes;
constexpr uint32_t kGemmSmem = kStages * kStageBytes + 1024;  // + alignment slack for the 1024-byte swizzle atoms
constexpr uint32_t kWaitLimit = 1u << 22;                     // polls (with back-off) before a wait gives up

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase of `parity` to complete.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (uint32_t i = 0; i < kWaitLimit; ++i) {
        if (mbar_test(bar, parity)) return true;
        if (i > 64) __nanosleep(32);
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, uint32_t x, uint32_t y,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor of a K-major tile with 128-byte swizzle:
// rows of 128 bytes (64 BF16 along K), 8-row atoms 1024 bytes apart (stride
// byte offset), descriptor version 1, layout type 2 (128-byte swizzle).
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16
// A and B (bits 7-9, 10-12 = 1), both K-major, N / 8 at bit 17, M / 16 at bit 24.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((kBN >> 3) << 17) | ((kBM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(kIdesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// ------------------------------------------------------------ prep kernel
// Row r of the group (one CTA per (job, loop), the FFT/select CTA map): the
// bucket sums z_l[j] (the job's gather partials summed in chunk order, as the
// FP32 path does), written as BF16 hi and lo parts of the interleaved row
// A[r] = (re z_0, im z_0, re z_1, ...): hi plane rows [0, Mpad), lo plane
// rows [Mpad, 2 Mpad).
__global__ void __launch_bounds__(kThreads) k_dft_prep(Launch ln, __nv_bfloat16 *A, uint32_t Mpad) {
    __shared__ PlanDev P;
    __shared__ Job J;
    __shared__ uint32_t s_local;
    enter(ln, P, J, s_local);
    const uint32_t l = s_local, B = P.B, row = blockIdx.x, nchunk = J.nchunk;
    const size_t cstride = (size_t)P.L * B;
    __nv_bfloat162 *hi = reinterpret_cast<__nv_bfloat162 *>(A + (size_t)row * 2 * B);
    __nv_bfloat162 *lo = reinterpret_cast<__nv_bfloat162 *>(A + ((size_t)Mpad + row) * 2 * B);
    for (uint32_t j = threadIdx.x; j < B; j += blockDim.x) {
        float2 acc = make_float2(0.f, 0.f);
        const float2 *src = P.partial + (size_t)l * B + j;
        for (uint32_t c = 0; c < nchunk; ++c) {
            const float2 v = __ldcg(src + c * cstride);
            acc.x += v.x;
            acc.y += v.y;
        }
        const __nv_bfloat162 h = __floats2bfloat162_rn(acc.x, acc.y);
        const float2 hf = __bfloat1622float2(h);
        hi[j] = h;
        lo[j] = __floats2bfloat162_rn(acc.x - hf.x, acc.y - hf.y);
    }
}

// ------------------------------------------------------------ GEMM kernel
// grid (Mpad / 128, 2B / 128, 3): tile (m0, n0) of product p (0: A_hi W_hi,
// 1: A_lo W_hi, 2: A_hi W_lo) into C[p][Mpad][2B] (FP32).
__global__ void __launch_bounds__(128, 1)
    k_dft_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmW, float *C,
               uint32_t Mpad, uint32_t twoB, uint32_t *err) {
    extern __shared__ uint8_t dsm[];
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages], accb;
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(dsm) + 1023) & ~(uintptr_t)1023);
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t m0 = blockIdx.x * kBM, n0 = blockIdx.y * kBN, p = blockIdx.z;
    const uint32_t nkb = twoB / kBK;  // k-blocks of one product
    const uint32_t ya = m0 + (p == 1 ? Mpad : 0u), yw = n0 + (p == 2 ? twoB : 0u);
    if (tid == 0) {
        for (uint32_t s = 0; s < kStages; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        mbar_init(smem_u32(&accb), 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(kBN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;

    if (tid == 0) {
        const uint32_t sbase = smem_u32(base);
        auto load = [&](uint32_t kb) {
            const uint32_t s = kb % kStages, a = sbase + s * kStageBytes;
            mbar_expect_tx(smem_u32(&full[s]), kStageBytes);
            tma_load_2d(a, &tmA, kb * kBK, ya, smem_u32(&full[s]));
            tma_load_2d(a + kTileBytes, &tmW, kb * kBK, yw, smem_u32(&full[s]));
        };
        const uint32_t pre = nkb < kStages ? nkb : kStages;
        for (uint32_t kb = 0; kb < pre; ++kb) load(kb);
        bool ok = true;
        for (uint32_t kb = 0; kb < nkb && ok; ++kb) {
            const uint32_t s = kb % kStages;
            if (!mbar_wait(smem_u32(&full[s]), (kb / kStages) & 1u)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a = sbase + s * kStageBytes;
            const uint64_t da = desc_sw128(a), dw = desc_sw128(a + kTileBytes);
#pragma unroll
            for (uint32_t k = 0; k < kBK / 16; ++k)  // 32 bytes along K per instruction
                mma_bf16(tmem, da + 2 * k, dw + 2 * k, (kb | k) != 0 ? 1u : 0u);
            mma_commit(smem_u32(&empty[s]));
            // refill the previous k-block's stage once its MMAs have read it
            if (kb >= 1 && kb - 1 + kStages < nkb) {
                const uint32_t sp = (kb - 1) % kStages;
                if (!mbar_wait(smem_u32(&empty[sp]), ((kb - 1) / kStages) & 1u)) {
                    ok = false;
                    break;
                }
                load(kb - 1 + kStages);
            }
        }
        if (!ok) {
            s_fail = 1;
            atomicExch(err, 1u);
        }
        mma_commit(smem_u32(&accb));  // arrives once every MMA issued above has completed
    }
    __syncthreads();
    // accumulator ready: every warp reads its 32 lanes (rows m0 + 32 warp + lane)
    const bool ready = mbar_wait(smem_u32(&accb), 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ready) atomicExch(err, 2u);
    const bool store = ready && !s_fail;
    float *dst = C + ((size_t)p * Mpad + m0 + 32 * warp + lane) * twoB + n0;
    for (uint32_t c = 0; c < kBN; c += 32) {
        uint32_t r[32];
        const uint32_t ta = tmem + ((32 * warp) << 16) + c;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
              "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
              "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
              "=r"(r[30]), "=r"(r[31])
            : "r"(ta));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (store) {
            float4 *d4 = reinterpret_cast<float4 *>(dst + c);
#pragma unroll
            for (uint32_t q = 0; q < 8; ++q)
                d4[q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                    __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kBN) : "memory");
}

// ------------------------------------------------------------ W table
// W^T in BF16, [2 planes][2B rows n][2B columns k]: plane 0 the hi parts,
// plane 1 the lo parts of W[k][n] (cos / sin from the exact turn (j k) mod B
// in FP64).
__global__ void k_dft_table(uint32_t B, __nv_bfloat16 *Wt) {
    const uint32_t twoB = 2 * B;
    const uint64_t total = (uint64_t)twoB * twoB;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t n = (uint32_t)(i / twoB), k = (uint32_t)(i % twoB);
        const uint32_t kk = n >> 1, co = n & 1, j = k >> 1, ci = k & 1;
        double sn, cs;
        sincospi(2.0 * (double)((uint64_t)j * kk % B) / (double)B, &sn, &cs);
        // row 2j + ci of W, column 2kk + co
        const double v = ci == 0 ? (co == 0 ? cs : -sn) : (co == 0 ? sn : cs);
        const __nv_bfloat16 h = __double2bfloat16(v);
        Wt[i] = h;
        Wt[total + i] = __double2bfloat16(v - (double)__bfloat162float(h));
    }
}

struct DftTable {
    int device;
    uint32_t B;
    __nv_bfloat16 *Wt;
    CUtensorMap map;
};

std::mutex g_dft_mu;
std::vector<DftTable> g_dft;

using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                              const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
    static EncodeFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
    });
    return fn;
}

// Tensor map of a [rows][2B] BF16 matrix (row stride 2B elements): boxes of
// 128 rows x 64 columns with 128-byte swizzle, zero fill out of range.
bool encode_rows(CUtensorMap *m, const void *ptr, uint32_t twoB, uint64_t rows) {
    EncodeFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {twoB, rows};
    const cuuint64_t strides[1] = {(cuuint64_t)twoB * 2};
    const cuuint32_t box[2] = {kBK, kBM};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

size_t dft_scratch_bytes(uint32_t rows, uint32_t B) {
    const size_t Mpad = ((size_t)rows + kBM - 1) / kBM * kBM;
    return Mpad * 2 * B * (2 * 2 + 3 * 4);  // A hi + lo (BF16), three FP32 partial planes
}

sfft_status dft_table_prepare(uint32_t B) {
    if (B < 64 || B > kDftMaxB || (B & (B - 1))) {
        set_error("precision 1 needs B a power of two in [64, 4096]");
        return SFFT_EINVAL;
    }
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lk(g_dft_mu);
    for (const DftTable &t : g_dft)
        if (t.device == device && t.B == B) return SFFT_OK;
    DftTable t{};
    t.device = device;
    t.B = B;
    const size_t n = (size_t)2 * (2 * B) * (2 * B);
    if ((e = cudaMalloc(&t.Wt, sizeof(__nv_bfloat16) * n)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(dft table)");
    cudaStream_t s = nullptr;
    if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) {
        cudaFree(t.Wt);
        return cuda_fail(e, "stream");
    }
    k_dft_table<<<1024, 256, 0, s>>>(B, t.Wt);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    if (e != cudaSuccess) {
        cudaFree(t.Wt);
        return cuda_fail(e, "dft table");
    }
    if (!encode_rows(&t.map, t.Wt, 2 * B, 2ull * 2 * B)) {
        cudaFree(t.Wt);
        set_error("cuTensorMapEncodeTiled failed for the DFT table");
        return SFFT_ECUDA;
    }
    g_dft.push_back(t);
    return SFFT_OK;
}

cudaError_t launch_dft(const Launch &ln, uint32_t rows, uint32_t B, void *scratch, uint32_t *err, cudaStream_t s) {
    if (rows == 0) return cudaSuccess;
    CUtensorMap wmap;
    {
        int device = 0;
        cudaError_t e = cudaGetDevice(&device);
        if (e != cudaSuccess) return e;
        std::lock_guard<std::mutex> lk(g_dft_mu);
        bool found = false;
        for (const DftTable &t : g_dft)
            if (t.device == device && t.B == B) {
                wmap = t.map;
                found = true;
            }
        if (!found) return cudaErrorInvalidValue;  // plans prepare their table at creation
    }
    const uint32_t Mpad = (rows + kBM - 1) / kBM * kBM, twoB = 2 * B;
    __nv_bfloat16 *A = static_cast<__nv_bfloat16 *>(scratch);
    float *C = reinterpret_cast<float *>(A + (size_t)2 * Mpad * twoB);
    CUtensorMap amap;
    if (!encode_rows(&amap, A, twoB, 2ull * Mpad)) return cudaErrorInvalidValue;
    k_dft_prep<<<rows, kThreads, 0, s>>>(ln, A, Mpad);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_dft_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemmSmem)) !=
        cudaSuccess)
        return e;
    k_dft_gemm<<<dim3(Mpad / kBM, twoB / kBN, 3), 128, kGemmSmem, s>>>(amap, wmap, C, Mpad, twoB, err);
    return cudaGetLastError();
}

const float *dft_partials(void *scratch, uint32_t rows, uint32_t B) {
    const uint32_t Mpad = (rows + kBM - 1) / kBM * kBM;
    return reinterpret_cast<const float *>(static_cast<__nv_bfloat16 *>(scratch) + (size_t)2 * Mpad * 2 * B);
}

}  // namespace sfft
