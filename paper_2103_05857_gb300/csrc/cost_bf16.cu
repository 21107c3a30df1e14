// cost_bf16.cu -- squared-Euclidean cost matrix on the 5th-generation tensor
// cores (tcgen05), for point clouds of feature dimension d >= 64:
//
//   C_ij = |x~_i|^2 + |y~_j|^2 - 2 <x~_i, y~_j>,
//
// x~, y~ = the points rounded to BF16 (round to nearest even), the inner
// products accumulated in FP32 in tensor memory, the norms of the rounded
// points summed in FP32. The paper's costs are Euclidean distances between
// colour centroids (Sec. 5.1); this GEMM form is the library's route for the
// squared cost of high-dimensional features.
//
// Kernel: persistent, one CTA per SM looping over 128 x 128 tiles of C, warp
// specialised. Warp 0 (one thread) streams the operands with TMA into a ring
// of four stages, each one 64-wide K block of the A (x~) and B (y~) tiles in
// the 128-byte-swizzled K-major layout. Warp 1 allocates tensor memory and
// (one thread) issues the tcgen05.mma (M = 128, N = 128, K = 16) of a tile
// into one of two 128-column FP32 accumulators, releasing each stage and
// then the accumulator through tcgen05.commit. Warps 2..9 are the epilogue,
// two per 32-lane quadrant of the accumulator, each taking half of the
// tile's columns: it reads its 32 lanes (tcgen05.ld 32x32b) in chunks of 32
// columns, hands the accumulator back, adds the norms, writes the chunk into
// one of three 128-byte-swizzled staging buffers and stores it with a TMA
// tensor store. So the next tile's loads and MMAs run under this tile's
// stores, and the store of C (the bound) streams without gaps.
//
// Every wait on an mbarrier is bounded; a wait that gives up sets an error
// flag the host reads, and the CTA still frees its tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace srot {

namespace {

constexpr int kBM = 128;             // rows of a tile (accumulator lanes)
constexpr int kBN = 128;             // columns of a tile (accumulator columns)
constexpr int kBK = 64;              // BF16 elements per 128-byte swizzle row
constexpr int kBoxBytes = kBM * 128; // one 128 x 64 BF16 box = 16 KiB
constexpr int kStages = 4;                 // operand ring: one K block per stage
constexpr int kStageOps = 2 * kBoxBytes;   // A and B boxes of one K block: 32 KiB
constexpr int kEpiWarps = 8;                 // two per accumulator lane quadrant
constexpr int kThreads = (2 + kEpiWarps) * 32;  // producer, MMA, epilogue warps
constexpr uint32_t kTmemCols = 2 * kBN;    // two accumulators
constexpr int kChunkBytes = 32 * 128;      // 32 rows x 32 FP32, one TMA store
constexpr int kStgChunks = 3;              // staging buffers per epilogue warp
constexpr size_t kSmemBytes =
    (size_t)kStages * kStageOps + (size_t)kEpiWarps * kStgChunks * kChunkBytes + 1024;
constexpr long long kSpinLimit = 1ll << 22;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Bounded wait for phase `parity` of an mbarrier; false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    for (long long it = 0; it < kSpinLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::
            "r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, int x, int y, const void *src) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];\n" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(smem_u32(src))
                 : "memory");
}

// Shared-memory matrix descriptor of a K-major operand in the 128-byte
// swizzled layout: rows of 128 bytes, groups of 8 rows 1024 bytes apart.
__device__ __forceinline__ uint64_t umma_desc_sw128(const void *p) {
    const uint64_t addr = smem_u32(p);
    uint64_t d = (addr & 0x3FFFFull) >> 4;  // start address
    d |= (uint64_t)1 << 16;                 // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                 // descriptor version
    d |= (uint64_t)2 << 61;                 // 128-byte swizzle
    return d;
}

// Instruction descriptor: BF16 x BF16 -> FP32, both operands K-major, M x N.
constexpr uint32_t umma_idesc_bf16(int M, int N) {
    return (1u << 4)                    // D: FP32
           | (1u << 7)                  // A: BF16
           | (1u << 10)                 // B: BF16
           | ((uint32_t)(N >> 3) << 17) // N / 8
           | ((uint32_t)(M >> 4) << 24);// M / 16
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld_32x32b_x32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

struct CostArgs {
    int m, n;
    int kb;           // d / 64
    const float *nx;  // m norms of the rounded points
    const float *ny;  // n
    int *err;         // set to 1 when a bounded wait gave up
};

__global__ void __launch_bounds__(kThreads, 1) k_cost_umma(const __grid_constant__ CUtensorMap tA,
                                                           const __grid_constant__ CUtensorMap tB,
                                                           const __grid_constant__ CUtensorMap tC, CostArgs P) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char *ops = smem;                              // kStages x {A box, B box}
    unsigned char *stg = smem + (size_t)kStages * kStageOps;  // epilogue warp e: 2 chunks
    __shared__ uint64_t full[kStages], empty[kStages], tfull[2], tempty[2];
    __shared__ uint32_t tmem_base_sh;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const unsigned FULL = 0xffffffffu;
    const int ntn = (P.n + kBN - 1) / kBN;
    const int ntiles = ((P.m + kBM - 1) / kBM) * ntn;

    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(&tmem_base_sh)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        for (int q = 0; q < kStages; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], 1);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(&tfull[q], 1);
            mbar_init(&tempty[q], kEpiWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;
    bool fail = false;

    if (warp == 0) {
        // ---- TMA producer: K blocks of this CTA's tiles into the ring
        if (lane == 0) {
            int kk = 0;
            for (int t = blockIdx.x; t < ntiles && !fail; t += gridDim.x) {
                const int m0 = (t / ntn) * kBM, n0 = (t % ntn) * kBN;
                for (int kbi = 0; kbi < P.kb; ++kbi, ++kk) {
                    const int q = kk % kStages;
                    const uint32_t ph = (uint32_t)(kk / kStages) & 1u;
                    if (!mbar_wait(&empty[q], ph ^ 1u)) { fail = true; break; }
                    unsigned char *sA = ops + (size_t)q * kStageOps;
                    mbar_expect_tx(&full[q], (uint32_t)kStageOps);
                    tma_load_2d(sA, &tA, kbi * kBK, m0, &full[q]);
                    tma_load_2d(sA + kBoxBytes, &tB, kbi * kBK, n0, &full[q]);
                }
            }
        }
    } else if (warp == 1) {
        // ---- MMA issuer: one tile into accumulator lt % 2
        if (lane == 0) {
            constexpr uint32_t idesc = umma_idesc_bf16(kBM, kBN);
            int kk = 0, lt = 0;
            for (int t = blockIdx.x; t < ntiles && !fail; t += gridDim.x, ++lt) {
                const int b = lt & 1;
                if (!mbar_wait(&tempty[b], ((uint32_t)(lt >> 1) & 1u) ^ 1u)) { fail = true; break; }
                tc_fence_after();
                const uint32_t td = tmem + (uint32_t)(b * kBN);
                for (int kbi = 0; kbi < P.kb; ++kbi, ++kk) {
                    const int q = kk % kStages;
                    if (!mbar_wait(&full[q], (uint32_t)(kk / kStages) & 1u)) { fail = true; break; }
                    tc_fence_after();
                    unsigned char *sA = ops + (size_t)q * kStageOps;
#pragma unroll
                    for (int s16 = 0; s16 < kBK / 16; ++s16)  // 16 BF16 = 32 bytes inside a swizzle row
                        umma_bf16(td, umma_desc_sw128(sA + 32 * s16), umma_desc_sw128(sA + kBoxBytes + 32 * s16),
                                  idesc, (kbi > 0 || s16 > 0) ? 1u : 0u);
                    umma_commit(&empty[q]);  // the stage is free once these MMAs have read it
                }
                if (fail) break;
                umma_commit(&tfull[b]);  // the accumulator is complete
            }
        }
    } else {
        // ---- epilogue: warp w reads accumulator lanes 32 (w % 4) .. + 31,
        // column chunks 2h, 2h + 1 with h = (w - 2) / 4
        const int qd = warp & 3, h = (warp - 2) >> 2;
        unsigned char *mystg = stg + (size_t)(warp - 2) * kStgChunks * kChunkBytes;
        int cb = 0, lt = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++lt) {
            const int b = lt & 1;
            int ok = 1;
            if (lane == 0) ok = mbar_wait(&tfull[b], (uint32_t)(lt >> 1) & 1u) ? 1 : 0;
            ok = __shfl_sync(FULL, ok, 0);
            if (!ok) { fail = true; break; }
            tc_fence_after();
            const int m0 = (t / ntn) * kBM, n0 = (t % ntn) * kBN;
            const int row = m0 + 32 * qd + lane;
            const float nxi = row < P.m ? __ldg(P.nx + row) : 0.f;
#pragma unroll 1
            for (int c = 2 * h; c < 2 * h + 2; ++c) {
                uint32_t r[32];
                tmem_ld_32x32b_x32(tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(b * kBN + 32 * c), r);
                if (c == 2 * h + 1) {  // this warp is done with the accumulator
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&tempty[b]);
                }
                // this staging buffer's previous store must have been read
                if (lane == 0) asm volatile("cp.async.bulk.wait_group.read %0;\n" ::"n"(kStgChunks - 1) : "memory");
                __syncwarp();
                float *chunk = reinterpret_cast<float *>(mystg + cb * kChunkBytes);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int j = n0 + 32 * c + 4 * u;  // n is a multiple of 4
                    const float4 yn = j < P.n ? __ldg(reinterpret_cast<const float4 *>(P.ny + j))
                                              : make_float4(0.f, 0.f, 0.f, 0.f);
                    float4 v;
                    v.x = fmaf(-2.f, __uint_as_float(r[4 * u + 0]), nxi + yn.x);
                    v.y = fmaf(-2.f, __uint_as_float(r[4 * u + 1]), nxi + yn.y);
                    v.z = fmaf(-2.f, __uint_as_float(r[4 * u + 2]), nxi + yn.z);
                    v.w = fmaf(-2.f, __uint_as_float(r[4 * u + 3]), nxi + yn.w);
                    // 128-byte swizzle: 16-byte unit u of row `lane` sits at unit u ^ (lane % 8)
                    *reinterpret_cast<float4 *>(chunk + lane * 32 + 4 * (u ^ (lane & 7))) = v;
                }
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                __syncwarp();
                if (lane == 0) {
                    tma_store_2d(&tC, n0 + 32 * c, m0 + 32 * qd, chunk);
                    asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
                }
                cb = cb + 1 == kStgChunks ? 0 : cb + 1;
            }
        }
        // the staging buffers may be released once the stores have read
        // them; their global writes complete with the grid
        if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
    }
    if (fail) atomicExch(P.err, 1);
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols));
    }
}

// Round to BF16 and FP32 norms of the rounded rows, X's m rows then Y's n
// rows in one launch; one warp per row.
__global__ void k_round_bf16(int m, int n, int d, const float *__restrict__ X, __nv_bfloat16 *__restrict__ Xb,
                             float *__restrict__ nx, const float *__restrict__ Y, __nv_bfloat16 *__restrict__ Yb,
                             float *__restrict__ ny, bool vec) {
    const int lane = threadIdx.x & 31;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int r = w; r < m + n; r += nw) {
        const bool isx = r < m;
        const int i = isx ? r : r - m;
        const float *src = isx ? X : Y;
        __nv_bfloat16 *dst = isx ? Xb : Yb;
        float s = 0.f;
        // d is a multiple of 64; with 16-byte aligned points every row starts
        // on a 16-byte boundary: four consecutive elements per lane
        for (int k = 4 * lane; vec && k < d; k += 4 * kWarp) {
            const float4 x = __ldg(reinterpret_cast<const float4 *>(src + (size_t)i * d + k));
            const __nv_bfloat162 lo = __floats2bfloat162_rn(x.x, x.y), hi = __floats2bfloat162_rn(x.z, x.w);
            uint2 pk;
            pk.x = *reinterpret_cast<const uint32_t *>(&lo);
            pk.y = *reinterpret_cast<const uint32_t *>(&hi);
            *reinterpret_cast<uint2 *>(dst + (size_t)i * d + k) = pk;
            const float2 flo = __bfloat1622float2(lo), fhi = __bfloat1622float2(hi);
            s = fmaf(flo.x, flo.x, s);
            s = fmaf(flo.y, flo.y, s);
            s = fmaf(fhi.x, fhi.x, s);
            s = fmaf(fhi.y, fhi.y, s);
        }
        for (int k = lane; !vec && k < d; k += kWarp) {
            const __nv_bfloat16 v = __float2bfloat16_rn(src[(size_t)i * d + k]);
            dst[(size_t)i * d + k] = v;
            const float f = __bfloat162float(v);
            s = fmaf(f, f, s);
        }
        s = warp_sum(s);
        if (lane == 0) (isx ? nx : ny)[i] = s;
    }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

bool encode_2d(CUtensorMap *map, CUtensorMapDataType dt, void *base, uint64_t inner, uint64_t outer,
               uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer) {
    std::call_once(g_encode_once, [] {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        else
            cudaGetLastError();
    });
    if (!g_encode) return false;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {row_bytes};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t estr[2] = {1, 1};
    return g_encode(map, dt, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

size_t cost_bf16_workspace(int m, int n, int d) {
    auto r = [](size_t b) { return ((b + 255) / 256) * 256; };
    return r((size_t)m * d * 2) + r((size_t)n * d * 2) + r((size_t)m * 4) + r((size_t)n * 4) + 256;
}

const char *launch_cost_bf16(int m, int n, int d, const float *X, const float *Y, float *C, void *ws,
                             int *err_dev, cudaStream_t st) {
    if (d % kBK != 0 || d < kBK || d > 256) return "d must be 64, 128, 192 or 256";
    if (n % 4 != 0) return "n must be a multiple of 4 (16-byte rows of C for the tensor store)";
    if (reinterpret_cast<uintptr_t>(C) % 16 != 0) return "C must be 16-byte aligned";
    auto r = [](size_t b) { return ((b + 255) / 256) * 256; };
    unsigned char *p = static_cast<unsigned char *>(ws);
    __nv_bfloat16 *Xb = reinterpret_cast<__nv_bfloat16 *>(p);
    p += r((size_t)m * d * 2);
    __nv_bfloat16 *Yb = reinterpret_cast<__nv_bfloat16 *>(p);
    p += r((size_t)n * d * 2);
    float *nx = reinterpret_cast<float *>(p);
    p += r((size_t)m * 4);
    float *ny = reinterpret_cast<float *>(p);

    const bool vec = reinterpret_cast<uintptr_t>(X) % 16 == 0 && reinterpret_cast<uintptr_t>(Y) % 16 == 0;
    k_round_bf16<<<std::min((m + n + 7) / 8, 152 * 8), 256, 0, st>>>(m, n, d, X, Xb, nx, Y, Yb, ny, vec);

    CUtensorMap tA, tB, tC;
    if (!encode_2d(&tA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, Xb, d, m, (uint64_t)d * 2, kBK, kBM) ||
        !encode_2d(&tB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, Yb, d, n, (uint64_t)d * 2, kBK, kBN) ||
        !encode_2d(&tC, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, C, n, m, (uint64_t)n * 4, 32, 32))
        return "tensor-map encoding failed";
    const int kb = d / kBK;
    static int sms = 0;  // persistent grid: one CTA per SM
    static bool attr_set = false;
    if (!attr_set) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 152;
        if (cudaFuncSetAttribute(k_cost_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes) !=
            cudaSuccess) {
            cudaGetLastError();
            return "shared-memory attribute rejected";
        }
        attr_set = true;
    }
    CostArgs P{m, n, kb, nx, ny, err_dev};
    const long long tiles = (long long)((m + kBM - 1) / kBM) * ((n + kBN - 1) / kBN);
    const int grid = (int)std::min<long long>(tiles, sms);
    k_cost_umma<<<grid, kThreads, kSmemBytes, st>>>(tA, tB, tC, P);
    return nullptr;
}

}  // namespace srot
