// batched.h -- the batched persistent solver's device-side descriptors.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace srot {

// One instance of a batch: sizes and element offsets into the packed arrays.
struct BatchInst {
    int m, n;
    long long off_X, off_Y, off_a, off_b, off_T, off_atoms;
};

// Per-instance outcome written by the kernel.
struct BatchResult {
    double f, g, feas;
    long long epochs, updates;
    int status;
    int pad;
};

enum InstStatus : int {
    kInstOk = 0,
    kInstNotConverged = 1,
    kInstNonFinite = 2,
    kInstNeedsDense = 3,  // a row outgrew its atom record: re-solve on the dense path
    kInstTimeout = 4,     // a bounded wait inside the epoch kernel gave up
};

struct BatchArgs {
    const BatchInst *inst;
    const int *queue;     // instance ids of this launch, largest first
    int queue_len;
    int *queue_head;      // work counter
    const float *X, *Y, *a, *b;
    float *T;
    int4 *atoms;
    BatchResult *res;
    double rho, tol;
    long long max_epochs;
    int gap_every;
    int variant, order, step;
    unsigned long long seed;
    int warm;             // 1: every instance starts from the plan in T
};

// ---------------------------------------------------------------------------
// Batched speculative form (solve_spec_batch.cu, solve_spec.cu in BATCH
// mode): one CTA per instance for the whole solve, each epoch the same as a
// single-instance speculative epoch, the certificate of Thm 2 taken inside
// the CTA when it is due. What an instance carries from one epoch to the next
// is in global memory: the plan, the atom records, the residual
// q = rho (s - b) in FP64 and this state.
// ---------------------------------------------------------------------------
struct SpecInstState {
    long long ep;         // epochs done
    long long updates;    // block updates done
    long long next_cert;  // epochs done before the next certificate may be taken
    double f, g, feas;    // last certificate
    double g_prev;        // gap at the last certificate that did not stop (0: none yet)
    long long ep_prev;    // epochs done at that certificate
    int active;           // 1 while the instance runs
    int status;           // InstStatus once stopped
    int devstat;          // DevStatus word of the epoch kernel (0: none)
    int resume;           // update at which a row outgrew its record, or -1
};

struct SpecBatchArgs {
    const BatchInst *inst;
    const int *list;      // instance ids of this launch, one per CTA (largest first)
    SpecInstState *state;
    double *q;            // per instance: rho (s - b), n doubles at the instance's b offset
    const float *X, *Y, *a, *b;
    float *T;
    int4 *atoms;
    double rho, tol;
    long long max_epochs;
    int gap_every;
    int warm;             // 1: every instance starts from the plan in T
};

constexpr int kSpecBatchMaxN = 4096;
constexpr int kSpecBatchBuckets = 2;
// Width bucket of an instance (n <= 2048 * 2^bucket), -1 above kSpecBatchMaxN.
int spec_batch_bucket(int n);
// Set-up of the instances list[0 .. count).
void launch_spec_batch_init(const SpecBatchArgs &B, int count, cudaStream_t st);
// The whole solve of the instances list[0 .. count) of one bucket; `uniform`
// selects uniform block order (else cyclic). False: the bucket is unknown.
bool launch_spec_batch_solve(int bucket, bool uniform, const SpecBatchArgs &B, int count,
                             unsigned long long seed, long long spin_limit, cudaStream_t st);

// Tile shapes of the batched kernel: ntc compute threads, g quads each, so
// an instance fits when n <= 4 * ntc * g.
struct BatchTile {
    int ntc, g;
};
extern const BatchTile kBatchTiles[];
extern const int kNumBatchTiles;

size_t batch_tile_smem(int t);
int batch_tile_ctas_per_sm(int t);
void launch_batched_tile(int t, const BatchArgs &B, int grid, cudaStream_t st);

}  // namespace srot
