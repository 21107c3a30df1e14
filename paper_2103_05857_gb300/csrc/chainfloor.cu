// chainfloor.cu -- the latency floor of the speculative epoch kernel's update
// chain (observability; not part of the paper's method).
//
// A block update of the speculative BCPFW kernel (solve_spec.cu) keeps on its
// dependent chain only what needs the residual left by the update before it:
// read the residual at the two columns that update changed, compare the two
// gradients with the prepared minimum, form the pairwise step (eq. 10) and
// write the residual of its own two columns back. This kernel runs exactly
// that chain, `updates` times, with nothing else: the same warp roles (one
// chain warp, or three in rotation handing over through "decided" and "done"
// mbarriers as the solver does), the same shared-memory residual words, the
// same compare-select and step arithmetic, and columns that change from one
// update to the next as a function of the previous decision (so no update can
// start before the one it depends on). Its time per update is the floor the
// solver's chain cannot go below with this hand-over design. Every wait is
// bounded; a wait that gives up sets *status.
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace srot {

namespace {

constexpr int kFloorCols = 4096;
constexpr int kFloorSlots = 8;
constexpr long long kFloorSpin = 1ll << 24;

__device__ inline unsigned fsaddr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ inline void fbar_init(uint64_t *b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(fsaddr(b)), "r"(count) : "memory");
}
__device__ inline void fbar_arrive(uint64_t *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(fsaddr(b)) : "memory");
}
__device__ inline bool fbar_try(uint64_t *b, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(fsaddr(b)), "r"(parity)
        : "memory");
    return done != 0;
}

template <int CH>
__global__ void __launch_bounds__(CH * 32, 1) k_chain_floor(int updates, int *status, float *sink) {
    __shared__ float qh[kFloorCols], ql[kFloorCols];
    __shared__ uint64_t decided[kFloorSlots], done[kFloorSlots];
    __shared__ int2 dec[kFloorSlots];
    __shared__ int stop;
    const int tid = threadIdx.x, lane = tid & 31, cw = tid >> 5;
    const unsigned FULL = 0xffffffffu;
    for (int j = tid; j < kFloorCols; j += CH * 32) {
        qh[j] = 1e-3f * (float)(j % 97);
        ql[j] = 0.f;
    }
    if (tid == 0) {
        for (int s = 0; s < kFloorSlots; ++s) {
            fbar_init(decided + s, 1);
            fbar_init(done + s, 1);
        }
        stop = 0;
    }
    __syncthreads();
    auto wait = [&](uint64_t *b, unsigned parity) -> bool {
        long long it = 0;
        while (!fbar_try(b, parity)) {
            if (*reinterpret_cast<volatile int *>(&stop)) return false;
            if (++it > kFloorSpin) {
                if (lane == 0) {
                    atomicCAS(status, 0, (int)kDevTimeout);
                    *reinterpret_cast<volatile int *>(&stop) = 1;
                }
                return false;
            }
        }
        return true;
    };
    const float a = 1.f / 4096.f, inv = 1.f / (2.f * 10.f * a), rho = 10.f;
    int2 mine = make_int2(1, 2);  // the columns the previous update of this warp changed (CH = 1)
    for (int u = cw; u < updates; u += CH) {
        const int slot = u % kFloorSlots;
        // prepared before the hand-over: the row's costs at two columns
        const float ce = 0.25f + 1e-4f * (float)((u * 37 + lane) & 255);
        int2 c1 = mine;
        if (CH > 1 && u >= 1) {
            const int ps = (u - 1) % kFloorSlots;
            const unsigned pp = (unsigned)((u - 1) / kFloorSlots) & 1u;
            if (!wait(decided + ps, pp)) break;
            c1 = dec[ps];
            if (!wait(done + ps, pp)) break;
        }
        // the residual at the two columns the previous update changed
        const int col = lane == 0 ? c1.x : c1.y;
        const float g = lane < 2 ? ce + qh[col] : 3.0e38f;
        const float g0 = __shfl_sync(FULL, g, 0), g1 = __shfl_sync(FULL, g, 1);
        const bool first = g0 <= g1;
        const int js = first ? c1.x : c1.y, v = first ? c1.y : c1.x;
        const float gmx = 0.5f + 1e-3f * (float)(u & 7);
        const float gam = fminf((fmaxf(g0, g1) - fminf(g0, g1)) * inv, gmx);
        // the columns this update changes: a function of the decision
        const int2 d = make_int2((js * 7 + u + 3) & (kFloorCols - 1), (v * 13 + u + 5) & (kFloorCols - 1));
        if (lane == 0) dec[slot] = d;
        __syncwarp();
        if (CH > 1 && lane == 0) fbar_arrive(decided + slot);
        // residual of this update's two columns (compensated, as the solver)
        if (lane < 2) {
            const int c = lane == 0 ? d.x : d.y;
            const float delta = (lane == 0 ? rho : -rho) * gam * a;
            const float y = __fsub_rn(delta, ql[c]);
            const float t = __fadd_rn(qh[c], y);
            ql[c] = __fsub_rn(__fsub_rn(t, qh[c]), y);
            qh[c] = t;
        }
        __syncwarp();
        if (CH > 1 && lane == 0) fbar_arrive(done + slot);
        mine = d;
    }
    __syncthreads();
    if (tid == 0) sink[0] = qh[0] + qh[kFloorCols - 1];
}

}  // namespace

void launch_chain_floor(int chain_warps, int updates, int *status, float *sink, cudaStream_t st) {
    if (chain_warps == 1) k_chain_floor<1><<<1, 32, 0, st>>>(updates, status, sink);
    else k_chain_floor<3><<<1, 96, 0, st>>>(updates, status, sink);
}

}  // namespace srot
