// solve_spec_batch.cu -- set-up of the batched speculative form (FP32,
// points with d = 3, pairwise steps).
//
// A batch solve in this form is one launch per width bucket of the
// speculative epoch kernel in BATCH mode (solve_spec.cu): CTA c owns
// instance list[c] for the whole solve and runs its epochs -- m block
// updates of Alg. A.3 with the exact line search (eq. 10), cyclic or uniform
// order, exactly as a single-instance epoch -- with the certificate of
// Thm 2 taken inside the CTA from the atom records when it is due
// (cert_records.cuh), until gap <= tol f with feasible rows or the epoch cap.
// The hardware schedules the CTAs (largest instances first), so instances
// never wait for one another. Before that launch, the set-up kernel below
// writes each instance's initial plan, atom records, residual q = rho (s - b)
// (FP64, exact column sums) and state.
#include <algorithm>
#include <limits>

#include "batched.h"
#include "cert_records.cuh"
#include "internal.h"

namespace srot {

namespace {

constexpr int kInitThreads = 256;

}  // namespace

// ---- set-up: T0 = (a_i e_0) (Thm 1) or the caller's plan, records, q --------
__global__ void __launch_bounds__(kInitThreads) k_spec_batch_init(SpecBatchArgs B) {
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long *csum = reinterpret_cast<unsigned long long *>(smem);
    __shared__ double red[kInitThreads / kWarp];
    __shared__ int sflag;
    const int inst = B.list[blockIdx.x];
    const BatchInst I = B.inst[inst];
    const int m = I.m, n = I.n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned FULL = 0xffffffffu;
    const float *a = B.a + I.off_a;
    float *T = B.T + I.off_T;
    int4 *grec = B.atoms + I.off_atoms;
    if (tid == 0) sflag = kInstOk;
    __syncthreads();
    if (!B.warm) {
        for (size_t e = tid; e < (size_t)m * n; e += kInitThreads) {
            const int i = (int)(e / n), j = (int)(e - (size_t)i * n);
            T[e] = j == 0 ? a[i] : 0.f;
        }
        for (int i = tid; i < m; i += kInitThreads) {
            const float ai = a[i];
            grec[(size_t)i * kAtomRecord] = make_int4(ai > 0.f ? 1 : 0, 0, 0, 0);
            grec[(size_t)i * kAtomRecord + 1] = make_int4(0, __float_as_int(ai), 0, 0);
        }
    } else {
        // the records of the caller's plan: each row's nonzero entries in
        // column order (one warp per row); a row with more than 63 stops the
        // instance for the dense path
        for (int i = warp; i < m; i += kInitThreads / kWarp) {
            const float *trow = T + (size_t)i * n;
            int4 *rec = grec + (size_t)i * kAtomRecord;
            int cnt = 0;
            for (int j0 = 0; j0 < n; j0 += kWarp) {
                const int j = j0 + lane;
                const float t = j < n ? trow[j] : 0.f;
                const unsigned mk = __ballot_sync(FULL, t > 0.f);
                const int pos = cnt + __popc(mk & ((1u << lane) - 1u));
                if (t > 0.f && pos < kAtomsMax) rec[1 + pos] = make_int4(j, __float_as_int(t), 0, 0);
                cnt += __popc(mk);
            }
            if (lane == 0) {
                rec[0] = make_int4(cnt <= kAtomsMax ? cnt : 0, 0, 0, 0);
                if (cnt > kAtomsMax) sflag = kInstNeedsDense;
            }
        }
    }
    __syncthreads();  // the records are written (global, this CTA)
    const int fx = rec_fixed_exp(rec_total_mass(a, m, red));
    rec_records_to_q(grec, m, n, B.b + I.off_b, B.rho, fx, csum);
    const double *q = reinterpret_cast<const double *>(csum);
    for (int j = tid; j < n; j += kInitThreads) B.q[I.off_b + j] = q[j];
    if (tid == 0) {
        SpecInstState S{};
        S.active = sflag == kInstOk ? 1 : 0;
        S.status = sflag;
        S.resume = -1;
        B.state[inst] = S;
    }
}

void launch_spec_batch_init(const SpecBatchArgs &B, int count, cudaStream_t st) {
    if (count <= 0) return;
    k_spec_batch_init<<<count, kInitThreads, 4096 * sizeof(unsigned long long), st>>>(B);
}

}  // namespace srot
