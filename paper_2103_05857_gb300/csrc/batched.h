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
