// common.cuh -- internal helpers shared by the library's translation units.
// Nothing here is part of the C ABI (include/sr_ot.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cfloat>
#include <cmath>

#include "../../include/sr_ot.h"

namespace srot {

constexpr int kWarp = 32;

// ---------------------------------------------------------------------------
// Device status word: kernels never trap; they record the first failure here
// and the host turns it into an sr_ot_status.
// ---------------------------------------------------------------------------
enum DevStatus : int {
    kDevOk = 0,
    kDevNonFinite = 1,   // a non-finite value met in an iterate
    kDevTimeout = 2,     // a bounded wait gave up
    kDevBadInput = 3,    // an input failed a device-side check
};

// ---------------------------------------------------------------------------
// splitmix64 (Steele, Lea & Flood, OOPSLA 2014): output number counter+1 of
// the generator seeded with seed ^ (stream << 56). Streams: 1 = permutation
// keys, 2 = uniform block draws, 3 = gap-adaptive draws.
// ---------------------------------------------------------------------------
__host__ __device__ inline uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
__host__ __device__ inline uint64_t sm64_draw(uint64_t seed, uint64_t stream, uint64_t counter) {
    return sm64_mix((seed ^ (stream << 56)) + (counter + 1ULL) * 0x9E3779B97F4A7C15ULL);
}
// floor(u * m) as the high word of the 128-bit product.
__device__ inline int scale_u64(uint64_t u, int m) {
    return (int)__umul64hi(u, (uint64_t)m);
}

// ---------------------------------------------------------------------------
// Order-preserving 32-bit keys for floats: key(a) < key(b) iff a < b for
// non-NaN a, b, after mapping -0 to +0.
// ---------------------------------------------------------------------------
__device__ inline uint32_t f2key(float v) {
    uint32_t u = __float_as_uint(v + 0.0f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ inline float key2f(uint32_t k) {
    uint32_t u = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
    return __uint_as_float(u);
}

// ---------------------------------------------------------------------------
// Exact FP64 arithmetic without contraction, for the bit-reproducible path.
// ---------------------------------------------------------------------------
__device__ inline double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ inline double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ inline double dmul(double a, double b) { return __dmul_rn(a, b); }

// Compensated (Kahan) FP32 accumulator; value() returns sum - comp in double,
// which carries the compensated result to about FP64 accuracy for the
// well-conditioned sums used here.
struct Kahan32 {
    float s = 0.f, c = 0.f;
    __device__ inline void add(float x) {
        // explicit round-to-nearest intrinsics: never contracted or reordered
        float y = __fsub_rn(x, c);
        float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ inline double value() const { return (double)s - (double)c; }
};

// Trace word 2 of a block update: the away vertex v in bits 0..28 (all ones
// when there is none) and the step's direction in bits 29..30 (0 toward the
// LMO vertex, 1 away from v, 2 pairwise, 3 no step).
__device__ inline int trace_vdir(int v, int kind) {
    const unsigned vv = v >= 0 ? ((unsigned)v & 0x1FFFFFFFu) : 0x1FFFFFFFu;
    const unsigned k = (kind >= 0 && kind <= 2) ? (unsigned)kind : 3u;
    return (int)(vv | (k << 29));
}

template <typename T>
__device__ inline T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace srot
