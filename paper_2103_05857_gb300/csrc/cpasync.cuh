// cpasync.cuh -- cp.async copies into shared memory and the (value, index)
// slot of the active-set kernels' argmin reduction.
#pragma once

#include <stdint.h>

namespace srot {

struct SpRed {
    uint32_t kmin;  // order-preserving key of the minimum
    int jmin;       // its column
};

__device__ inline void cp16(void *smem_dst, const void *gsrc) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc));
}
__device__ inline void cp4(void *smem_dst, const void *gsrc) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc));
}
__device__ inline void commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ inline void wait_groups() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

}  // namespace srot
