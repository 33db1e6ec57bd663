// bn_persistent.h — launch interface of the persistent, SMEM-blocked sweep kernel.
#pragma once

#include "bn_device.cuh"

namespace bn {

// Grid barrier state; zeroed before every launch.
struct GridBarrier {
    unsigned int count;
    unsigned int gen;
    unsigned int error;
    unsigned int pad;
};

// ~1 s at 2 GHz: a barrier wait longer than this records an error and the kernel returns.
constexpr long long kBarrierSpinCycles = 1ll << 31;

constexpr int kMaxTsplit = 4;  // chunk ranges per block (side_cls holds 2 x kMaxTsplit parts)

struct PersistentArgs {
    const Problem *probs;   // device array
    int n_prob;
    const int *unit_start;  // [n_prob + 1] prefix sums of work units per problem
    const int *couple_start;// [n_prob + 1] prefix sums of couples per problem
    int total_units, total_couples;
    int tsplit;
    int n_iter;             // passes in this launch (problems stop at their own pass end)
    GridBarrier *bar;
    int *work;              // [2] unit counters of phase 1, by pass parity; zeroed per launch
};

// CTA shape: block of bx x by pixels, threads per CTA, proposed pixels per warp per round
struct PersistentShape {
    int bx, by, threads, spw, tsplit;
};

// Instantiated CTA shapes: X(bx, by, compute warps, proposed pixels per warp per round, min
// CTAs per SM); every CTA has one more warp, the producer (threads = 32 * (compute warps + 1)).
#define BN_PERSISTENT_SHAPES(X) \
    X(8, 8, 7, 4, 2)            \
    X(16, 8, 15, 4, 1)          \
    X(8, 16, 15, 4, 1)

int persistent_units_per_problem(const Problem &h, int bx, int by, int tsplit);
bool persistent_supported(const Problem &h);
bool persistent_shape_fits(const Problem &h, const PersistentShape &s);
cudaError_t launch_persistent(const PersistentArgs &a, const PersistentShape &shape, int cb,
                              int sms, cudaStream_t st);
cudaError_t launch_fold_error(const GridBarrier *gb, const Problem *probs, int n_prob,
                              cudaStream_t st);
cudaError_t launch_selftest_wait(int which, long long budget, GridBarrier *gb, int *result,
                                 cudaStream_t st);

}  // namespace bn
