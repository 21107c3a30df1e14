// solve_spec.cu -- one epoch of BCPFW (pairwise steps, Alg. A.3, exact line
// search eq. 10) on a single instance with d = 3 points, cyclic or permuted
// block order, the heavy per-row work of the next updates done ahead of the
// update chain.
//
// A pairwise step of row i changes the residual in two columns only (the LMO
// vertex j* and the away vertex v). So the statistics of a later row can be
// taken against an older residual and repaired: for update u, producer warps
// take the minimum of C_ij + q_j over their own segment of columns, and the
// atom warp the away vertex (maximum of the gradient over the row's atoms),
// each with the residual as it stood after `ver` updates, ver >= u - kSpecLag.
// When the chain warp reaches update u it knows which columns changed since
// (a per-column index of the last update that changed it, and the columns of
// the last kSpecLag updates in registers):
//   - a segment minimum whose column has not changed since ver is exact for
//     every unchanged column of its segment;
//   - every column changed in the last kSpecLag updates is evaluated with the
//     current residual (one per lane);
//   - a segment whose minimum sits on a changed column is recomputed in full,
//     and so are the away statistics if one of the row's atoms changed (both
//     rare).
// The minimum over these, ties to the smallest column, is the exact LMO. All
// decisions equal those of the two-phase kernel (solve_sparse.cu) bit for bit.
//
// Warps 0..NWP-1 produce segment minima (their columns: quads tid + NTC g),
// warps NWP, NWP+1 (atom warps, even and odd updates) stream the atom
// records, take the away statistics and publish the row's data, warps
// NWP+2 .. NWP+1+CH are the chain (update u goes to warp u mod CH; with
// CH = 3, while one warp decides and applies an update, the next prepares
// its own; with CH = 1 one warp prepares, decides and applies). They
// synchronise through mbarriers only (no polling): per slot a "full" barrier
// on which the producers and the atom warp arrive (release) once their words
// for update u are stored and on which the chain waits (acquire), and per
// update a "done" barrier on which the chain arrives once the residual of
// update u is in shared memory (before the update's global stores, so the
// release never waits on them) and on which producers wait before reading
// the residual for update u + kSpecLag + 1. Every wait is bounded.
#include <algorithm>
#include <climits>
#include <limits>

#include "atoms.cuh"
#include "batched.h"
#include "cert_records.cuh"
#include "common.cuh"
#include "cpasync.cuh"
#include "internal.h"
#include "step.cuh"

namespace srot {

namespace {

constexpr int kSmemMax = 227 * 1024;
constexpr int kSpecLag = 4;        // producers run at most this many updates ahead of the chain
constexpr int kSpecSlots = 8;      // candidate / atom-warp slots (> kSpecLag)
constexpr int kSpecRecAhead = 4;   // atom records are fetched this many updates early
constexpr int kSpecRecSlots = 16;  // record slots (> kSpecLag + kSpecRecAhead)
constexpr int kSpecRecHead = 8;    // record entries fetched ahead: the count and 7 atoms (128 bytes);
                                   // a row with more atoms has the rest copied when it is used
// Chain warps CH: 3 (warp c takes the updates u = c mod 3, the hand-over
// takes the columns of u-2, then those of u-1) or 1 (one warp takes every
// update; it knows every column changed since the producers' residual
// without waiting on another warp).
constexpr long long kSpecSpin = 1ll << 26;  // default polls before a wait gives up
constexpr int kGcAhead = 2;                 // given cost: rows a producer thread has in flight
constexpr int kGcRing = kGcAhead + 1;       // and its row slots in shared memory
static_assert(kSpecSlots > kSpecLag && kSpecRecSlots > kSpecLag + kSpecRecAhead, "slot rings too small");
static_assert(kSpecRecSlots * kAtomRecord * 4 >= kRecRowChunk, "the certificate's row chunk lives in the record ring");

__device__ inline unsigned saddr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ inline int vload(const int *p) { return *reinterpret_cast<const volatile int *>(p); }
__device__ inline void vstore(int *p, int v) { *reinterpret_cast<volatile int *>(p) = v; }
__device__ inline void mbar_init(uint64_t *b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(saddr(b)), "r"(count) : "memory");
}
__device__ inline void mbar_inval(uint64_t *b) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(saddr(b)) : "memory");
}
__device__ inline void mbar_arrive(uint64_t *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(saddr(b)) : "memory");
}
// One bounded probe of phase `parity` (the hardware may suspend the warp
// for a while before it answers false).
__device__ inline bool mbar_try(uint64_t *b, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(saddr(b)), "r"(parity)
        : "memory");
    return done != 0;
}
constexpr int kAtomWords = 3;  // atom warp output per update: int4 words


}  // namespace

// BATCH: CTA c solves instance Bt.list[c] of a batch (its sizes and arrays
// from the batch descriptors, the other settings from A0): epoch after epoch,
// the barriers re-initialised between them, the certificate of Thm 2 taken
// inside the CTA when it is due, until the instance stops.
// GC: the cost matrix C is given (row-major m x n, rows on 16-byte
// boundaries, n a multiple of 4) instead of the points: the producers load
// their segment of each row ahead of the residual gate, the other warps read
// the entries they need (a few per update) from global memory.
template <int NWP, int G, int CH, bool SPLIT, bool BATCH, bool GC>
__global__ void __launch_bounds__(NWP * kWarp + (2 + CH) * kWarp, (BATCH && G <= 4) ? 2 : 1)
    k_epoch_spec(EpochArgs<float> A0, SpecBatchArgs Bt) {
    constexpr int NTC = NWP * kWarp;  // producer threads
    constexpr int AW = NWP;  // atom warps NWP, NWP + 1; chain warps NWP + 2 ...
    constexpr int NT = NTC + (2 + CH) * kWarp;
    constexpr int WID = NTC * 4 * G;
    static_assert(CH == 1 || CH == 3, "one chain warp, or three in rotation");
    static_assert(!SPLIT || CH == 3, "the split chain has two preparer warps and one decider");
    static_assert(CH <= kSpecLag, "the changed columns are known for the updates ver .. u-1");
    static_assert(WID <= 8192, "column index must fit the 14 bits of the atom word");
    static_assert(!(GC && BATCH), "the batched form takes points");
    static_assert(NWP + 2 * (kSpecLag - CH + 1) <= kWarp, "candidates and changed columns must fit one warp");
    extern __shared__ __align__(16) unsigned char smem[];
    float *qh = reinterpret_cast<float *>(smem);
    float *ql = qh + WID;
    float4 *ys = reinterpret_cast<float4 *>(ql + WID);
    int *lastmod = reinterpret_cast<int *>(ys + (GC ? 0 : WID));  // last update that changed column j
    int4 *aring = reinterpret_cast<int4 *>(lastmod + WID);       // kSpecRecSlots atom records
    int4 *aw = aring + (size_t)kSpecRecSlots * kAtomRecord;       // kSpecSlots x kAtomWords
    unsigned long long *cand = reinterpret_cast<unsigned long long *>(aw + kSpecSlots * kAtomWords);  // kSpecSlots x NWP
    uint64_t *full = reinterpret_cast<uint64_t *>(cand + kSpecSlots * NWP);  // kSpecSlots
    uint64_t *done = full + kSpecSlots;                                      // kSpecSlots
    uint64_t *decided = done + kSpecSlots;                                   // kSpecSlots
    uint64_t *prepd = decided + kSpecSlots;                                  // kSpecSlots (split chain)
    int2 *dec = reinterpret_cast<int2 *>(prepd + kSpecSlots);                // columns update u changes
    int4 *prep = reinterpret_cast<int4 *>(dec + kSpecSlots);                 // prepared words (split chain)
    int *ctl = reinterpret_cast<int *>(prep + kSpecSlots);                   // [0] stop
    int *recent = ctl + 4;                                                   // rows of the last 16 updates
    double *cred = reinterpret_cast<double *>(recent + 16);                  // certificate partials (BATCH)
    float *cring = reinterpret_cast<float *>(cred + 6 * 16);                 // GC: kGcRing rows of C

    EpochArgs<float> A = A0;
    int inst = -1;
    const float *bvec = nullptr;
    if constexpr (BATCH) {
        inst = Bt.list[blockIdx.x];
        if (!Bt.state[inst].active) return;  // uniform over the CTA
        const BatchInst I = Bt.inst[inst];
        A.in.m = I.m;
        A.in.n = I.n;
        A.in.X = Bt.X + I.off_X;
        A.in.Y = Bt.Y + I.off_Y;
        A.in.a = Bt.a + I.off_a;
        A.T = Bt.T + I.off_T;
        A.q = Bt.q + I.off_b;
        A.atoms = Bt.atoms + I.off_atoms;
        A.status = &Bt.state[inst].devstat;
        A.resume = &Bt.state[inst].resume;
        A.k0 = Bt.state[inst].ep * (long long)I.m;
        bvec = Bt.b + I.off_b;
    }
    // a row outgrew its atom record in an earlier epoch: the dense kernel
    // takes every epoch from now on (its records are no longer kept)
    if (A.sticky && *reinterpret_cast<const volatile int *>(A.sticky)) {
        if (threadIdx.x == 0 && A.resume) *A.resume = 0;
        return;
    }
    const int m = A.in.m, n = A.in.n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned FULL = 0xffffffffu;
    const float rho = (float)A.rho;
    const int order = A.order;
    int4 *grec = A.atoms;
    const float INF = std::numeric_limits<float>::infinity();
    int fx = 0;  // BATCH: fixed-point scale of the certificate's column sums
    if constexpr (BATCH) fx = rec_fixed_exp(rec_total_mass(A.in.a, m, cred));
    // BATCH: the certificate of the current plan (all threads); q refreshed
    // in global memory; the instance's state updated; true to stop
    auto certify = [&](long long E) -> bool {
        unsigned long long *csum = reinterpret_cast<unsigned long long *>(qh);  // WID words over qh, ql
        float *qf = reinterpret_cast<float *>(lastmod);  // reset before the next epoch
        int *jrow = reinterpret_cast<int *>(aring);        // kSpecRecSlots x 1 KiB = kRecRowChunk ints
        const RecCert c = rec_certificate(grec, m, n, A.in.X, ys, A.in.a, bvec, Bt.rho, fx, csum, qf, jrow, cred);
        const double *qd = reinterpret_cast<const double *>(csum);
        for (int j = tid; j < n; j += NT) A.q[j] = qd[j];
        if (tid == 0) {
            SpecInstState &S = Bt.state[inst];
            S.f = c.f;
            S.g = c.g;
            S.feas = c.feas;
            const bool conv = Bt.tol > 0.0 && c.g <= Bt.tol * c.f && c.feas <= kFeasTol;
            int stop = 0;
            if (conv || E >= Bt.max_epochs) {
                S.status = (conv || Bt.tol <= 0.0) ? kInstOk : kInstNotConverged;
                S.active = 0;
                stop = 1;
            } else if (Bt.tol > 0.0) {
                // the next certificate when the gap's decay since the last one,
                // taken as geometric (linear convergence), predicts the
                // tolerance; at most 8 epochs on (each refreshes the residual)
                long long skip = 2;
                if (S.g_prev > 0.0 && c.g > 0.0 && c.g < S.g_prev && E > S.ep_prev) {
                    const double rate = log(c.g / S.g_prev) / (double)(E - S.ep_prev);  // < 0
                    const double need = log(Bt.tol * c.f / c.g) / rate;                  // > 0
                    const double early = 0.75 * need;  // rather a certificate too early than late
                    skip = early >= 8.0 ? 8 : (early < 1.0 ? 1 : (long long)early);
                }
                S.g_prev = c.g;
                S.ep_prev = E;
                S.next_cert = E + skip * Bt.gap_every;
            }
            ctl[1] = stop;
        }
        __syncthreads();
        return ctl[1] != 0;
    };
    bool finished = false;
    if constexpr (BATCH) {
        if (Bt.max_epochs <= 0) {  // the certificate of the initial plan only
            for (int j = tid; j < n; j += NT)
                ys[j] = make_float4(A.in.Y[(size_t)j * 3], A.in.Y[(size_t)j * 3 + 1], A.in.Y[(size_t)j * 3 + 2], 0.f);
            __syncthreads();
            finished = certify(0);
            finished = true;
        }
    }

    // ---- epochs: one per launch, or (BATCH) until the instance stops -----
    for (int epoch_in_launch = 0; !finished; ++epoch_in_launch) {
    for (int j = tid; j < WID; j += NT) {
        if (j < n) {
            const double qq = A.q[j];
            const float h = (float)qq;
            qh[j] = h;
            ql[j] = (float)((double)h - qq);
            if (!GC)
                ys[j] = make_float4(A.in.Y[(size_t)j * 3], A.in.Y[(size_t)j * 3 + 1], A.in.Y[(size_t)j * 3 + 2], 0.f);
        } else {
            qh[j] = 1e30f;
            ql[j] = 0.f;
            if (!GC) ys[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        lastmod[j] = -1;
    }
    const long long spin = A.spin_limit > 0 ? A.spin_limit : kSpecSpin;
    if (tid == 0) {
        for (int s = 0; s < kSpecSlots; ++s) {
            if (epoch_in_launch > 0) {  // every wait and arrival of the last epoch is over
                mbar_inval(full + s);
                mbar_inval(done + s);
                mbar_inval(decided + s);
                mbar_inval(prepd + s);
            }
            mbar_init(full + s, NWP + 1);
            mbar_init(done + s, 1);
            mbar_init(decided + s, 1);
            mbar_init(prepd + s, 1);
            dec[s] = make_int2(-1, -1);
        }
        ctl[0] = 0;
        if (SPLIT)
            for (int e = 0; e < 16; ++e) recent[e] = -1;
        if (A.resume) *A.resume = -1;
        if (A.gate) {  // the start gate: a bounded wait for a non-zero word
            long long it = 0;
            while (vload(A.gate) == 0) {
                if (++it > spin) {
                    atomicCAS(A.status, 0, (int)kDevTimeout);
                    ctl[0] = 1;
                    break;
                }
                __nanosleep(64);
            }
        }
    }
    __syncthreads();
    const bool gate_closed = ctl[0] != 0;  // every warp skips its loop

    auto row_of = [&](int u) -> int {
        if (order == SR_OT_PERMUTE) return A.perm[u];
        // uniform order runs on the split chain only
        if (SPLIT && order == SR_OT_UNIFORM) return scale_u64(sm64_draw(A.seed, 2, (uint64_t)(A.k0 + u)), m);
        return u;
    };
    // gradient of row x (points) or of the row of C at crow (GC) at column j
    // with the residual as it is now
    auto grad_at = [&](int j, float x0, float x1, float x2, const float *crow) -> float {
        if constexpr (GC) {
            return (j < n ? __ldg(crow + j) : 0.f) + qh[j];  // padding columns: qh = 1e30
        } else {
            const float4 y = ys[j];
            const float d0 = x0 - y.x, d1 = x1 - y.y, d2 = x2 - y.z;
            return fmaf(d2, d2, fmaf(d1, d1, __fmul_rn(d0, d0))) + qh[j];
        }
    };
    auto crow_of = [&](int row) -> const float * { return GC ? A.in.C + (size_t)row * n : nullptr; };
    // producers and the atom warp: wait until the chain has applied update
    // u - kSpecLag - 1 (its residual is then visible); false to stop
    auto gate = [&](int u) -> bool {
        const int p = u - kSpecLag - 1;
        if (p < 0) return true;
        long long it = 0;
        while (!mbar_try(done + p % kSpecSlots, (unsigned)(p / kSpecSlots) & 1u)) {
            if (vload(ctl)) return false;
            if (++it > spin) {
                if (lane == 0) {
                    atomicCAS(A.status, 0, (int)kDevTimeout);
                    vstore(ctl, 1);
                }
                return false;
            }
        }
        return true;
    };
    // x and a of the rows of this warp's next two updates (loaded early)
    float xa[2][4];
    auto load_xa = [&](int s, int u) {
        xa[s][0] = xa[s][1] = xa[s][2] = xa[s][3] = 0.f;
        if (u < m) {
            const int i = row_of(u);
            if (!GC) {
                xa[s][0] = A.in.X[(size_t)i * 3];
                xa[s][1] = A.in.X[(size_t)i * 3 + 1];
                xa[s][2] = A.in.X[(size_t)i * 3 + 2];
            }
            xa[s][3] = A.in.a[i];
        }
    };
    auto shift_xa = [&] {
#pragma unroll
        for (int e = 0; e < 4; ++e) xa[0][e] = xa[1][e];
    };

    if (gate_closed) {
        // the start gate timed out: no update is made, the residual is kept
    } else if (warp < NWP) {
        // ================= producers: segment minima =====================
        float2 ny0[GC ? 1 : 2 * G], ny1[GC ? 1 : 2 * G], ny2[GC ? 1 : 2 * G];
        if constexpr (!GC) {
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int j = 4 * (tid + NTC * g) + 2 * h;
                    const float4 ya = ys[j], yb = ys[j + 1];
                    ny0[2 * g + h] = make_float2(-ya.x, -yb.x);
                    ny1[2 * g + h] = make_float2(-ya.y, -yb.y);
                    ny2[2 * g + h] = make_float2(-ya.z, -yb.z);
                }
        }
        load_xa(0, 0);
        load_xa(1, 1);
        // GC: each thread copies its own columns of the rows kGcAhead updates
        // ahead into its part of a ring of rows (cp.async, L2 only), so the
        // HBM latency of a row is hidden behind the updates before it
        auto fetch_row = [&](int t) {
            if (t < m) {
                const float *crow = crow_of(row_of(t));
                float *dst = cring + (size_t)(t % kGcRing) * WID;
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    const int j0 = 4 * (tid + NTC * g);
                    if (j0 < n) cp16(dst + j0, crow + j0);
                }
            }
            commit();
        };
        if constexpr (GC)
            for (int t = 0; t < kGcAhead; ++t) fetch_row(t);
        for (int u = 0; u < m; ++u) {
            float4 cv[GC ? G : 1];
            if constexpr (GC) {
                fetch_row(u + kGcAhead);
                wait_groups<kGcAhead>();  // row u has landed (this thread's own copies)
                const float *src = cring + (size_t)(u % kGcRing) * WID;
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    const int j0 = 4 * (tid + NTC * g);
                    cv[g] = j0 < n ? *reinterpret_cast<const float4 *>(src + j0) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            if (!gate(u)) break;
            const float2 X0 = make_float2(xa[0][0], xa[0][0]), X1 = make_float2(xa[0][1], xa[0][1]),
                         X2 = make_float2(xa[0][2], xa[0][2]);
            float qv[G];
            int qj[G];
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const int j0 = 4 * (tid + NTC * g);
                const float4 q4 = *reinterpret_cast<const float4 *>(qh + j0);
                float2 c[2];
                if constexpr (GC) {
                    c[0] = make_float2(cv[g].x, cv[g].y);
                    c[1] = make_float2(cv[g].z, cv[g].w);
                } else {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const float2 d0 = __fadd2_rn(X0, ny0[2 * g + h]), d1 = __fadd2_rn(X1, ny1[2 * g + h]),
                                     d2 = __fadd2_rn(X2, ny2[2 * g + h]);
                        float2 cc = __fmul2_rn(d0, d0);
                        cc = __ffma2_rn(d1, d1, cc);
                        c[h] = __ffma2_rn(d2, d2, cc);
                    }
                }
                const float2 ga = __fadd2_rn(c[0], make_float2(q4.x, q4.y));
                const float2 gb = __fadd2_rn(c[1], make_float2(q4.z, q4.w));
                const bool ta = ga.y < ga.x, tb = gb.y < gb.x;
                const float va = ta ? ga.y : ga.x, vb = tb ? gb.y : gb.x;
                const int ia = j0 + (ta ? 1 : 0), ib = j0 + (tb ? 3 : 2);
                const bool tq = vb < va;
                qv[g] = tq ? vb : va;
                qj[g] = tq ? ib : ia;
            }
#pragma unroll
            for (int w = 1; w < G; w <<= 1)
#pragma unroll
                for (int g = 0; g + w < G; g += 2 * w)
                    if (qv[g + w] < qv[g]) { qv[g] = qv[g + w]; qj[g] = qj[g + w]; }
            const uint32_t km = f2key(qv[0]);
            const uint32_t wk = __reduce_min_sync(FULL, km);
            const int wj = __reduce_min_sync(FULL, km == wk ? qj[0] : 0x7FFFFFFF);
            if (lane == 0) {
                cand[(u % kSpecSlots) * NWP + warp] = (unsigned long long)wk | ((unsigned long long)wj << 32);
                mbar_arrive(full + u % kSpecSlots);
            }
            shift_xa();
            load_xa(1, u + 2);
        }
        if constexpr (GC) wait_groups<0>();  // no copy in flight at exit
    } else if (warp < AW + 2) {
        // ============ two atom warps (even, odd updates): records, away
        // ============ statistics, row data
        const int aw0 = warp - AW;
        auto fetch_record = [&](int t) {
            if (t < m && lane < kSpecRecHead) {
                const int i = row_of(t);
                int4 *dst = aring + (size_t)(t % kSpecRecSlots) * kAtomRecord;
                cp16(dst + lane, grec + (size_t)i * kAtomRecord + lane);
            }
            commit();
        };
        fetch_record(aw0);
        fetch_record(aw0 + 2);
        load_xa(0, aw0);
        load_xa(1, aw0 + 2);
        // GC: the cost entries of the next update's head atoms (lane l: atom
        // l < 7), loaded one iteration of this warp before their use
        float pc = 0.f;
        int pcj = -1;
        auto prefetch_c = [&](int t) {
            pcj = -1;
            if (GC && t < m) {
                const int4 *r = aring + (size_t)(t % kSpecRecSlots) * kAtomRecord;
                if (lane < r[0].x && lane < kSpecRecHead - 1) {
                    pcj = r[1 + lane].x;
                    pc = __ldg(crow_of(row_of(t)) + pcj);
                }
            }
        };
        if constexpr (GC) {
            wait_groups<1>();  // the head of update aw0's record
            __syncwarp();
            prefetch_c(aw0);
        }
        for (int u = aw0; u < m; u += 2) {
            if (!gate(u)) break;
            wait_groups<1>();  // the head of update u's record has landed (u + 2's may be in flight)
            __syncwarp();
            int4 *rs = aring + (size_t)(u % kSpecRecSlots) * kAtomRecord;
            {
                const int cnt = rs[0].x;  // warp-uniform
                if (cnt >= kSpecRecHead) {
                    // more atoms than the head holds (rare): copy the rest now;
                    // the row's record is not written again before update u
                    const int4 *src = grec + (size_t)row_of(u) * kAtomRecord;
                    for (int e = kSpecRecHead + lane; e <= cnt && e < kAtomRecord; e += kWarp) rs[e] = src[e];
                    __syncwarp();
                }
            }
            const float x0 = xa[0][0], x1 = xa[0][1], x2 = xa[0][2], au = xa[0][3];
            LaneAtoms at = load_atoms(rs, lane);
            DF tvd{0.f, 0.f};
            const float *crow = crow_of(row_of(u));
            auto grad = [&](int j) -> float {
                if constexpr (GC) return (j == pcj ? pc : __ldg(crow + j)) + qh[j];
                else return grad_at(j, x0, x1, x2, crow);
            };
            const AtomStats st = atom_stats(at, grad, au, false, &tvd);
            if (lane == 0) {
                const float ra = au > 0.f ? 1.f / au : 0.f;
                const float ia = au > 0.f ? 1.f / (2.f * rho * au) : 0.f;
                const int vv = (st.v >= 0 && st.v < n) ? st.v : 0x3FFF;
                int4 *o = aw + (u % kSpecSlots) * kAtomWords;
                o[0] = make_int4(__float_as_int(st.gmax), __float_as_int(tvd.hi), __float_as_int(tvd.lo),
                                 vv | ((st.vpos + 1) << 14));
                o[1] = make_int4(__float_as_int(x0), __float_as_int(x1), __float_as_int(x2), __float_as_int(au));
                o[2] = make_int4(__float_as_int(ra), __float_as_int(ia), row_of(u), 0);
                mbar_arrive(full + u % kSpecSlots);
            }
            if constexpr (GC) {
                wait_groups<0>();  // the head of update u + 2's record
                __syncwarp();
                prefetch_c(u + 2);
            }
            fetch_record(u + kSpecRecAhead);
            shift_xa();
            load_xa(1, u + 4);
        }
        wait_groups<0>();
    } else if (SPLIT && warp < AW + 4) {
        // ================= split chain: two preparer warps ================
        // Preparer (u mod 2) takes everything of update u that does not need
        // the residual of u-3, u-2 and u-1: once update u-4 is published, the
        // segment minima (recomputed where their column changed since ver),
        // the columns changed by updates ver..u-4, the record position of
        // the likely vertex and whether an atom changed since ver. The
        // decider merges the columns of u-3, u-2 and u-1 itself.
        const int pw = warp - (NWP + 2);
        auto wait_bar = [&](uint64_t *b, unsigned parity) -> bool {
            long long it = 0;
            while (!mbar_try(b, parity)) {
                if (vload(ctl)) return false;
                if (++it > spin) {
                    if (lane == 0) {
                        atomicCAS(A.status, 0, (int)kDevTimeout);
                        vstore(ctl, 1);
                    }
                    return false;
                }
            }
            return true;
        };
        for (int u = pw; u < m; u += 2) {
            const int slot = u % kSpecSlots;
            if (u >= 4) {
                const int p4 = u - 4;
                if (!wait_bar(done + p4 % kSpecSlots, (unsigned)(p4 / kSpecSlots) & 1u)) break;
            }
            if (!wait_bar(full + slot, (unsigned)(u / kSpecSlots) & 1u)) break;
            const unsigned long long cw = lane < NWP ? cand[slot * NWP + lane] : 0ull;
            const int4 w1 = aw[slot * kAtomWords + 1];
            const int ver = u > kSpecLag ? u - kSpecLag : 0;
            const float x0 = __int_as_float(w1.x), x1 = __int_as_float(w1.y), x2 = __int_as_float(w1.z);
            LaneAtoms at = load_atoms(aring + (size_t)(u % kSpecRecSlots) * kAtomRecord, lane);
            const float *crow = crow_of(aw[slot * kAtomWords + 2].z);
            auto grad = [&](int j) -> float { return grad_at(j, x0, x1, x2, crow); };
            uint32_t key = 0xFFFFFFFFu;
            int col = 0x7FFFFFFF;
            bool stale = false;
            if (lane < NWP) {
                const int cj = (int)(cw >> 32);
                stale = lastmod[cj] >= ver;
                if (!stale) {
                    key = (uint32_t)cw;
                    col = cj;
                }
            } else if (lane < NWP + 2 * (kSpecLag - 3)) {
                const int w = u - 4 - ((lane - NWP) >> 1);
                if (w >= ver && w >= 0) {
                    const int2 d = dec[w % kSpecSlots];
                    const int c = ((lane - NWP) & 1) ? d.y : d.x;
                    if (c >= 0) {
                        key = f2key(grad(c));
                        col = c;
                    }
                }
            }
            unsigned fb = __ballot_sync(FULL, stale);
            while (fb) {
                const int w = __ffs(fb) - 1;
                fb &= fb - 1;
                float bv = INF;
                int bj = 0x7FFFFFFF;
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    const int j0 = 4 * (kWarp * w + lane + NTC * g);
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float gv = grad(j0 + e);
                        if (gv < bv) { bv = gv; bj = j0 + e; }
                    }
                }
                const uint32_t kb = f2key(bv);
                const uint32_t wk = __reduce_min_sync(FULL, kb);
                const int wj = __reduce_min_sync(FULL, kb == wk ? bj : 0x7FFFFFFF);
                if (lane == w) { key = wk; col = wj; }
            }
            const uint32_t pk = __reduce_min_sync(FULL, key);
            const int pj = __reduce_min_sync(FULL, key == pk ? col : 0x7FFFFFFF);
            const bool olddirty = __any_sync(FULL, (at.j[0] >= 0 && lastmod[at.j[0]] >= ver) ||
                                                       (at.cnt > 32 && at.j[1] >= 0 && lastmod[at.j[1]] >= ver));
            bool present = false;
            int jpos = -1;
            atom_weight(at, pj, &present, &jpos);
            if (lane == 0) {
                prep[slot] = make_int4((int)pk, pj, olddirty ? 1 : 0, jpos);
                mbar_arrive(prepd + slot);
            }
        }
    } else if (SPLIT) {
        // ================= split chain: the decider =======================
        // One warp decides and applies every update. It knows the columns
        // the last three updates changed (its own), merges their exact keys
        // with the prepared minimum in one warp reduction (the full LMO
        // instead when that minimum sits on one of them), takes the away
        // statistics again when one of the row's atoms changed, decides,
        // applies and publishes -- with no hand-over between warps on its
        // chain.
        bool aborted = false;
        int c1[2] = {-1, -1}, c2[2] = {-1, -1}, c3[2] = {-1, -1};  // columns of updates u-1, u-2, u-3
        const bool repeats = order == SR_OT_UNIFORM;  // a row may come back within the window
        for (int u = 0; u < m; ++u) {
            const long long k = A.k0 + u;
            const int slot = u % kSpecSlots;
            {
                long long it = 0;
                while (!mbar_try(prepd + slot, (unsigned)(u / kSpecSlots) & 1u)) {
                    if (vload(ctl)) { aborted = true; break; }
                    if (++it > spin) {
                        if (lane == 0) {
                            atomicCAS(A.status, 0, (int)kDevTimeout);
                            vstore(ctl, 1);
                        }
                        aborted = true;
                        break;
                    }
                }
                if (aborted) break;
            }
            const int4 pr = prep[slot];
            const uint32_t pk = (uint32_t)pr.x;
            const int pj = pr.y;
            const bool olddirty = pr.z != 0;
            int jpos = pr.w;
            bool present = jpos >= 0;
            const int4 w0 = aw[slot * kAtomWords], w1 = aw[slot * kAtomWords + 1], w2 = aw[slot * kAtomWords + 2];
            const int row = w2.z;
            const float x0 = __int_as_float(w1.x), x1 = __int_as_float(w1.y), x2 = __int_as_float(w1.z);
            const float ai = __int_as_float(w1.w), ra = __int_as_float(w2.x), ia = __int_as_float(w2.y);
            LaneAtoms at = load_atoms(aring + (size_t)(u % kSpecRecSlots) * kAtomRecord, lane);
            // uniform order: if the row was updated in the last 12 updates, the
            // record was fetched before that update stored it: read it again
            // (this warp stored it) and retake everything taken from it
            bool fresh = false;
            if (repeats) {
                fresh = __any_sync(FULL, lane < 12 && u - 1 - lane >= 0 && recent[(u - 1 - lane) & 15] == row);
                if (fresh) {
                    __syncwarp();
                    at = load_atoms(grec + (size_t)row * kAtomRecord, lane);
                    present = false;
                    jpos = -1;
                    atom_weight(at, pj, &present, &jpos);
                }
                __syncwarp();
                if (lane == 0) recent[u & 15] = row;
            }
            const float *crow = crow_of(row);
            auto grad = [&](int j) -> float { return grad_at(j, x0, x1, x2, crow); };
            // the columns of updates u-1, u-2, u-3 (lanes 0..5) join the
            // prepared minimum (lane 6); a prepared minimum on one of them was
            // taken at a residual that has changed since: the full LMO instead
            const int hc = lane < 6 ? ((lane >> 1) == 0 ? c1[lane & 1] : (lane >> 1) == 1 ? c2[lane & 1] : c3[lane & 1])
                                    : -1;
            const bool redo_lmo = __any_sync(FULL, hc >= 0 && hc == pj);
            uint32_t fk = pk;
            int js = pj;
            const int pj2 = pj;
            auto hit = [&](int c) {
                return c >= 0 && (c == c1[0] || c == c1[1] || c == c2[0] || c == c2[1] || c == c3[0] || c == c3[1]);
            };
            const bool redo_atoms =
                __any_sync(FULL, fresh || olddirty || hit(at.j[0]) || (at.cnt > 32 && hit(at.j[1])));
            if (!redo_lmo) {
                uint32_t ke = 0xFFFFFFFFu;
                int ce = 0x7FFFFFFF;
                if (hc >= 0) {
                    ke = f2key(grad(hc));
                    ce = hc;
                } else if (lane == 6) {
                    ke = pk;
                    ce = pj;
                }
                fk = __reduce_min_sync(FULL, ke);
                js = __reduce_min_sync(FULL, ke == fk ? ce : 0x7FFFFFFF);
            }
            if (redo_lmo) {
                float bv = INF;
                int bj = 0x7FFFFFFF;
                for (int q = lane; q < WID / 4; q += kWarp) {
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float gv = grad(4 * q + e);
                        if (gv < bv) { bv = gv; bj = 4 * q + e; }
                    }
                }
                const uint32_t kb = f2key(bv);
                fk = __reduce_min_sync(FULL, kb);
                js = __reduce_min_sync(FULL, kb == fk ? bj : 0x7FFFFFFF);
            }
            const float gmin = key2f(fk);
            DF tvd{__int_as_float(w0.y), __int_as_float(w0.z)};
            AtomStats st;
            if (redo_atoms) {
                st = atom_stats(at, grad, ai, false, &tvd);
            } else {
                const int v14 = w0.w & 0x3FFF;
                st.v = v14 == 0x3FFF ? 0x7FFFFFFF : v14;
                st.vpos = (w0.w >> 14) - 1;
                st.gmax = __int_as_float(w0.x);
                st.t_v = tvd.hi;
                st.nnz = at.cnt;
                st.g_aw = st.s2 = st.dda = 0.f;
            }
            if (!isfinite(gmin)) {
                if (lane == 0) atomicCAS(A.status, 0, (int)kDevNonFinite);
                aborted = true;
                break;
            }
            float gmx = 0.f, inv = 0.f;
            if (ai > 0.f) {
                gmx = st.t_v * ra;  // same rounding as the two-phase kernel
                inv = ia;
            }
            if (js != pj2) atom_weight(at, js, &present, &jpos);
            const Step<float> S = decide_pairwise(st, gmin, js, ai, rho, gmx, inv, n);
            const bool moved = S.kind == 2 && S.v != S.js && st.vpos >= 0;
            if (lane == 0) dec[slot] = moved ? make_int2(S.js, S.v) : make_int2(-1, -1);
            auto publish = [&] {
                if (lane == 0 && moved) {
                    lastmod[S.js] = u;
                    lastmod[S.v] = u;
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(done + slot);
            };
            const bool ok = apply_pairwise(S, at, jpos, st.vpos, tvd, rho, A.T + (size_t)row * n, qh, ql,
                                           grec + (size_t)row * kAtomRecord, lane, publish);
            if (!ok) {  // j* would be a 64th atom: the dense kernel takes over at u
                if (lane == 0 && A.resume) *A.resume = u;
                if (lane == 0 && A.sticky) *A.sticky = 1;
                aborted = true;
                break;
            }
            if (lane == 0 && A.trace && k < A.trace_cap) {
                A.trace[4 * k] = row;
                A.trace[4 * k + 1] = js;
                A.trace[4 * k + 2] = trace_vdir((st.v >= 0 && st.v < n) ? st.v : -1, S.kind);
                A.trace[4 * k + 3] = __float_as_int(S.gamma);
            }
            c3[0] = c2[0];
            c3[1] = c2[1];
            c2[0] = c1[0];
            c2[1] = c1[1];
            c1[0] = moved ? S.js : -1;
            c1[1] = moved ? S.v : -1;
        }
        if (aborted && lane == 0) vstore(ctl, 1);  // releases every other warp still waiting
    } else {
        // ================= chain warps ====================================
        // Warp NWP + 2 + (u mod CH) takes update u. It prepares u
        // (segment minima, the columns changed by updates ver..u-CH, the
        // away statistics) while the other chain warps decide and apply the
        // updates before it; then it merges the columns that u-2 changed
        // (decided and stored an update earlier), takes the two that u-1
        // changes once u-1 is decided, waits until their residual is stored,
        // evaluates them and decides.
        const int cwi = warp - (NWP + 2);
        bool aborted = false;
        auto wait_bar = [&](uint64_t *b, unsigned parity) -> bool {
            long long it = 0;
            while (!mbar_try(b, parity)) {
                if (vload(ctl)) return false;
                if (++it > spin) {
                    if (lane == 0) {
                        atomicCAS(A.status, 0, (int)kDevTimeout);
                        vstore(ctl, 1);
                    }
                    return false;
                }
            }
            return true;
        };
        for (int u = cwi; u < m; u += CH) {
            const long long k = A.k0 + u;
            const int slot = u % kSpecSlots;
            const int ps = (u + kSpecSlots - 1) % kSpecSlots;  // slot of update u - 1
            const unsigned pp = u >= 1 ? (unsigned)((u - 1) / kSpecSlots) & 1u : 0u;
            // ---- prepare ------------------------------------------------
            if (!wait_bar(full + slot, (unsigned)(u / kSpecSlots) & 1u)) { aborted = true; break; }
            const unsigned long long cw = lane < NWP ? cand[slot * NWP + lane] : 0ull;
            const int4 w0 = aw[slot * kAtomWords], w1 = aw[slot * kAtomWords + 1], w2 = aw[slot * kAtomWords + 2];
            const int row = w2.z;
            const int ver = u > kSpecLag ? u - kSpecLag : 0;  // residual age of every word of update u
            const float x0 = __int_as_float(w1.x), x1 = __int_as_float(w1.y), x2 = __int_as_float(w1.z);
            const float ai = __int_as_float(w1.w), ra = __int_as_float(w2.x), ia = __int_as_float(w2.y);
            // the atom warp's copy of the record (ordered by the full barrier)
            LaneAtoms at = load_atoms(aring + (size_t)(u % kSpecRecSlots) * kAtomRecord, lane);
            const float *crow = crow_of(row);
            // GC: the cost entries of row u at the likely columns of update
            // u-1 (its segment minima and away vertex as prepared, and the
            // columns of u-3, which it merges), loaded now so that the
            // columns u-1 changes are found here after the hand-over
            float pcv = 0.f, hcv = 0.f;
            int pcx = -1, hcx = -1;
            if constexpr (GC) {
                if (u >= 1) {
                    const int sp = (u - 1) % kSpecSlots;
                    if (lane < NWP) {
                        pcx = (int)(cand[sp * NWP + lane] >> 32);
                    } else if (lane == NWP) {
                        const int v14 = aw[sp * kAtomWords].w & 0x3FFF;  // may still be filling: only a guess
                        pcx = v14 == 0x3FFF ? -1 : v14;
                    } else if (lane < NWP + 3 && u >= 3) {
                        const int2 d = dec[(u - 3) % kSpecSlots];
                        pcx = lane == NWP + 1 ? d.x : d.y;
                    }
                    if (pcx >= 0 && pcx < n) pcv = __ldg(crow + pcx);
                    else pcx = -1;
                }
            }
            auto grad = [&](int j) -> float { return grad_at(j, x0, x1, x2, crow); };
            // clean segment minima and the columns changed by updates ver..u-2
            uint32_t key = 0xFFFFFFFFu;
            int col = 0x7FFFFFFF;
            bool stale = false;
            if (lane < NWP) {
                const int cj = (int)(cw >> 32);
                stale = lastmod[cj] >= ver;
                if (!stale) {
                    key = (uint32_t)cw;
                    col = cj;
                }
            } else if (lane < NWP + 2 * (kSpecLag - CH + 1)) {
                const int w = u - CH - ((lane - NWP) >> 1);
                if (w >= ver && w >= 0) {
                    const int2 d = dec[w % kSpecSlots];
                    const int c = ((lane - NWP) & 1) ? d.y : d.x;
                    if (c >= 0) {
                        key = f2key(grad(c));
                        col = c;
                    }
                }
            }
            unsigned fb = __ballot_sync(FULL, stale);
            while (fb) {
                const int w = __ffs(fb) - 1;
                fb &= fb - 1;
                float bv = INF;
                int bj = 0x7FFFFFFF;
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    const int j0 = 4 * (kWarp * w + lane + NTC * g);
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float gv = grad(j0 + e);
                        if (gv < bv) { bv = gv; bj = j0 + e; }
                    }
                }
                const uint32_t kb = f2key(bv);
                const uint32_t wk = __reduce_min_sync(FULL, kb);
                const int wj = __reduce_min_sync(FULL, kb == wk ? bj : 0x7FFFFFFF);
                if (lane == w) { key = wk; col = wj; }
            }
            const uint32_t pk = __reduce_min_sync(FULL, key);
            const int pj = __reduce_min_sync(FULL, key == pk ? col : 0x7FFFFFFF);
            const bool olddirty = (at.j[0] >= 0 && lastmod[at.j[0]] >= ver) ||
                                  (at.cnt > 32 && at.j[1] >= 0 && lastmod[at.j[1]] >= ver);
            // the record position of the likely vertex pj (off the hand-over)
            bool present = false;
            int jpos = -1;
            atom_weight(at, pj, &present, &jpos);
            // ---- hand-over, 1: update u-2, decided and stored an update
            // earlier: the exact keys of its two columns join the prepared
            // minimum (a prepared minimum on one of them was stale: the full
            // LMO is taken instead)
            int c2[2] = {-1, -1}, c1[2] = {-1, -1};
            if (CH > 1 && u >= 2) {
                const int s2 = (u - 2) % kSpecSlots;
                const unsigned p2 = (unsigned)((u - 2) / kSpecSlots) & 1u;
                if (!wait_bar(decided + s2, p2) || !wait_bar(done + s2, p2)) { aborted = true; break; }
                const int2 d = dec[s2];
                c2[0] = d.x;
                c2[1] = d.y;
            }
            bool redo_lmo = pj >= 0 && (pj == c2[0] || pj == c2[1]);
            uint32_t fk = pk;
            int js = pj;
            {
                const int c = lane == 0 ? c2[0] : c2[1];
                uint32_t ke = 0xFFFFFFFFu;
                if (lane < 2 && c >= 0) {
                    if constexpr (GC) {  // kept for the hand-over of u-1 (its columns may be these)
                        hcx = c;
                        hcv = __ldg(crow + c);
                        ke = f2key(hcv + qh[c]);
                    } else {
                        ke = f2key(grad(c));
                    }
                }
                const uint32_t k0 = __shfl_sync(FULL, ke, 0), k1 = __shfl_sync(FULL, ke, 1);
                if (c2[0] >= 0 && (k0 < fk || (k0 == fk && c2[0] < js))) { fk = k0; js = c2[0]; }
                if (c2[1] >= 0 && (k1 < fk || (k1 == fk && c2[1] < js))) { fk = k1; js = c2[1]; }
            }
            const int pj2 = js;
            if (pj2 != pj) atom_weight(at, pj2, &present, &jpos);
            // ---- hand-over, 2: update u-1, its columns, then their residual
            if (CH > 1 && u >= 1) {
                if (!wait_bar(decided + ps, pp)) { aborted = true; break; }
                const int2 d = dec[ps];
                c1[0] = d.x;
                c1[1] = d.y;
            }
            redo_lmo = redo_lmo || (pj2 >= 0 && (pj2 == c1[0] || pj2 == c1[1]));
            auto hit = [&](int c) { return c >= 0 && (c == c1[0] || c == c1[1] || c == c2[0] || c == c2[1]); };
            const bool redo_atoms = __any_sync(FULL, olddirty || hit(at.j[0]) || (at.cnt > 32 && hit(at.j[1])));
            // what does not depend on the residual of u-1: the cost of the
            // row at its two columns (lanes 0, 1)
            const int ec = lane == 0 ? c1[0] : c1[1];
            float ce = 0.f;
            if constexpr (GC) {
                // the cost at the columns of u-1 from the entries loaded ahead,
                // else (rarely) from memory
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int c = c1[e];
                    const unsigned ma = __ballot_sync(FULL, c >= 0 && pcx == c);
                    const unsigned mb = __ballot_sync(FULL, c >= 0 && hcx == c);
                    const float va = __shfl_sync(FULL, pcv, ma ? __ffs(ma) - 1 : 0);
                    const float vb = __shfl_sync(FULL, hcv, mb ? __ffs(mb) - 1 : 0);
                    const float v = ma ? va : (mb ? vb : (c >= 0 ? __ldg(crow + c) : 0.f));
                    if (lane == e) ce = v;
                }
            }
            if (lane < 2 && ec >= 0) {
                if constexpr (GC) {
                } else {
                    const float4 y = ys[ec];
                    const float d0 = x0 - y.x, d1 = x1 - y.y, d2 = x2 - y.z;
                    ce = fmaf(d2, d2, fmaf(d1, d1, __fmul_rn(d0, d0)));
                }
            }
            if (CH > 1 && u >= 1 && !wait_bar(done + ps, pp)) { aborted = true; break; }
            if (redo_lmo) {
                // the prepared minimum sits on a column changed since: full LMO
                float bv = INF;
                int bj = 0x7FFFFFFF;
                for (int q = lane; q < WID / 4; q += kWarp) {
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float gv = grad(4 * q + e);
                        if (gv < bv) { bv = gv; bj = 4 * q + e; }
                    }
                }
                const uint32_t kb = f2key(bv);
                fk = __reduce_min_sync(FULL, kb);
                js = __reduce_min_sync(FULL, kb == fk ? bj : 0x7FFFFFFF);
            } else {
                const uint32_t ke = (lane < 2 && ec >= 0) ? f2key(ce + qh[ec]) : 0xFFFFFFFFu;
                const uint32_t k0 = __shfl_sync(FULL, ke, 0), k1 = __shfl_sync(FULL, ke, 1);
                if (c1[0] >= 0 && (k0 < fk || (k0 == fk && c1[0] < js))) { fk = k0; js = c1[0]; }
                if (c1[1] >= 0 && (k1 < fk || (k1 == fk && c1[1] < js))) { fk = k1; js = c1[1]; }
            }
            const float gmin = key2f(fk);
            DF tvd{__int_as_float(w0.y), __int_as_float(w0.z)};
            AtomStats st;
            if (redo_atoms) {
                st = atom_stats(at, grad, ai, false, &tvd);
            } else {
                const int v14 = w0.w & 0x3FFF;
                st.v = v14 == 0x3FFF ? 0x7FFFFFFF : v14;
                st.vpos = (w0.w >> 14) - 1;
                st.gmax = __int_as_float(w0.x);
                st.t_v = tvd.hi;
                st.nnz = at.cnt;
                st.g_aw = st.s2 = st.dda = 0.f;
            }
            if (!isfinite(gmin)) {
                if (lane == 0) atomicCAS(A.status, 0, (int)kDevNonFinite);
                aborted = true;
                break;
            }
            float gmx = 0.f, inv = 0.f;
            if (ai > 0.f) {
                gmx = st.t_v * ra;  // same rounding as the two-phase kernel
                inv = ia;
            }
            if (js != pj2) atom_weight(at, js, &present, &jpos);
            const Step<float> S = decide_pairwise(st, gmin, js, ai, rho, gmx, inv, n);
            // ---- decision of u: the columns it changes, for the other warp
            const bool moved = S.kind == 2 && S.v != S.js && st.vpos >= 0;
            if (lane == 0) dec[slot] = moved ? make_int2(S.js, S.v) : make_int2(-1, -1);
            __syncwarp();
            if (CH > 1 && lane == 0) mbar_arrive(decided + slot);
            // after the residual has changed: release of update u, before the
            // plan entries and the record are stored
            auto publish = [&] {
                if (lane == 0 && moved) {
                    lastmod[S.js] = u;
                    lastmod[S.v] = u;
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(done + slot);
            };
            const bool ok = apply_pairwise(S, at, jpos, st.vpos, tvd, rho, A.T + (size_t)row * n, qh, ql,
                                           grec + (size_t)row * kAtomRecord, lane, publish);
            if (!ok) {  // j* would be a 64th atom: the dense kernel takes over at u
                if (lane == 0 && A.resume) *A.resume = u;
                if (lane == 0 && A.sticky) *A.sticky = 1;
                aborted = true;
                break;
            }
            if (lane == 0 && A.trace && k < A.trace_cap) {
                A.trace[4 * k] = row;
                A.trace[4 * k + 1] = js;
                A.trace[4 * k + 2] = trace_vdir((st.v >= 0 && st.v < n) ? st.v : -1, S.kind);
                A.trace[4 * k + 3] = __float_as_int(S.gamma);
            }
        }
        if (aborted && lane == 0) vstore(ctl, 1);  // releases every other warp still waiting
    }
    __syncthreads();
    for (int j = tid; j < n; j += NT) A.q[j] = (double)qh[j] - (double)ql[j];
    if constexpr (!BATCH) {
        break;
    } else {
        // count the epoch; stop on a record overflow, a non-finite value or
        // a wait that gave up; else take the certificate when it is due
        if (tid == 0) {
            SpecInstState &S = Bt.state[inst];
            const int rs = *A.resume, ds = *A.status;
            S.ep += 1;
            S.updates += rs >= 0 ? rs : m;
            int stop = 0, due = 0;
            if (rs >= 0 || ds != 0) {
                S.status = rs >= 0 ? kInstNeedsDense : (ds == kDevTimeout ? kInstTimeout : kInstNonFinite);
                S.active = 0;
                stop = 1;
            } else {
                const long long E = S.ep;
                due = (E % Bt.gap_every == 0 && E >= S.next_cert) || E >= Bt.max_epochs;
            }
            ctl[1] = stop;
            ctl[2] = due;
            ctl[3] = (int)(S.ep & 0x7FFFFFFF);
        }
        __syncthreads();
        if (ctl[1]) break;
        if (ctl[2] && certify(Bt.state[inst].ep)) break;
        A.k0 += m;
    }
    }  // epochs
}

template <int NWP, int G, bool GC = false>
static size_t spec_smem() {
    constexpr int WID = NWP * kWarp * 4 * G;
    size_t b = (size_t)WID * (4 + 4 + (GC ? 0 : 16) + 4);
    if (GC) b += (size_t)kGcRing * WID * 4;
    b += (size_t)kSpecRecSlots * kAtomRecord * 16;
    b += (size_t)kSpecSlots * (kAtomWords * 16 + NWP * 8 + 4 * 8 + 8 + 16);
    b += 16 + 16 * 4 + 6 * 16 * sizeof(double);
    return b;
}

template <int NWP, int G, int CH, bool SPLIT, bool BATCH = false, bool GC = false>
static void launch_spec(const EpochArgs<float> &A, cudaStream_t st, const SpecBatchArgs *B = nullptr,
                        int grid = 1) {
    auto kern = k_epoch_spec<NWP, G, CH, SPLIT, BATCH, GC>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax);
        attr_set = true;
    }
    SpecBatchArgs none{};
    kern<<<grid, NWP * kWarp + (2 + CH) * kWarp, spec_smem<NWP, G, GC>(), st>>>(A, B ? *B : none);
}

template <int CH, bool SPLIT>
static bool launch_spec_ch(const EpochArgs<float> &A, cudaStream_t st) {
    const int n = A.in.n;
    if (n <= 128 * 4) launch_spec<4, 1, CH, SPLIT>(A, st);
    else if (n <= 128 * 8) launch_spec<4, 2, CH, SPLIT>(A, st);
    else if (n <= 128 * 16) launch_spec<4, 4, CH, SPLIT>(A, st);
    else if (n <= 128 * 32) launch_spec<4, 8, CH, SPLIT>(A, st);
    else return false;
    return true;
}

int spec_batch_bucket(int n) {
    for (int b = 0; b < kSpecBatchBuckets; ++b)
        if (n <= 2048 << b) return b;
    return -1;
}

template <bool SPLIT>
static bool launch_spec_batch_b(int bucket, const EpochArgs<float> &A, const SpecBatchArgs &B, int count,
                                cudaStream_t st) {
    // one instantiation for every n <= 2048: CTAs of different kernels on
    // one SM slowed each other's chains far more than two of the same code
    // (measured at 2048-column tiles: 1.21x for a pair of one kernel, above
    // 2x for a 2048-wide and a 512-wide kernel side by side)
    switch (bucket) {
        case 0: launch_spec<4, 4, 3, SPLIT, true>(A, st, &B, count); return true;
        case 1: launch_spec<4, 8, 3, SPLIT, true>(A, st, &B, count); return true;
        default: return false;
    }
}

bool launch_spec_batch_solve(int bucket, bool uniform, const SpecBatchArgs &B, int count,
                             unsigned long long seed, long long spin_limit, cudaStream_t st) {
    if (count <= 0) return true;
    EpochArgs<float> A{};
    A.in.cost_mode = kCostPts3;
    A.rho = B.rho;
    A.variant = SR_OT_BCPFW;
    A.step = SR_OT_ELS;
    A.order = uniform ? SR_OT_UNIFORM : SR_OT_CYCLIC;
    A.seed = seed;
    A.spin_limit = spin_limit;
    return uniform ? launch_spec_batch_b<true>(bucket, A, B, count, st)
                   : launch_spec_batch_b<false>(bucket, A, B, count, st);
}

// Given cost: three chain warps in rotation, cyclic or permuted order, n a
// multiple of 4 up to 8192 with 16-byte aligned rows.
static bool launch_spec_given(const EpochArgs<float> &A, cudaStream_t st) {
    const int n = A.in.n;
    if (!A.vec || (n % 4) != 0) return false;
    if (A.order != SR_OT_CYCLIC && A.order != SR_OT_PERMUTE) return false;
    if (n <= 128 * 4) launch_spec<4, 1, 3, false, false, true>(A, st);
    else if (n <= 128 * 8) launch_spec<4, 2, 3, false, false, true>(A, st);
    else if (n <= 128 * 16) launch_spec<4, 4, 3, false, false, true>(A, st);
    else if (n <= 128 * 32) launch_spec<4, 8, 3, false, false, true>(A, st);
    else if (n <= 128 * 64) launch_spec<4, 16, 3, false, false, true>(A, st);
    else return false;
    return true;
}

bool launch_epoch_spec(const EpochArgs<float> &A, cudaStream_t st, int chain) {
    if (A.variant != SR_OT_BCPFW) return false;
    if (A.in.cost_mode == kCostGiven) return chain == 3 && launch_spec_given(A, st);
    if (A.in.cost_mode != kCostPts3) return false;
    if (chain == kSpecChainSplit) {
        if (A.order != SR_OT_CYCLIC && A.order != SR_OT_PERMUTE && A.order != SR_OT_UNIFORM) return false;
        return launch_spec_ch<3, true>(A, st);
    }
    if (A.order != SR_OT_CYCLIC && A.order != SR_OT_PERMUTE) return false;
    return chain == 1 ? launch_spec_ch<1, false>(A, st) : launch_spec_ch<3, false>(A, st);
}

}  // namespace srot
