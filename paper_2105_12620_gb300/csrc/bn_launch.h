// bn_launch.h — host-side launchers of the sampler's kernels (internal to the library).
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "bn_device.cuh"
#include "bn_sample.cuh"
#include "bn_sampler.h"

namespace bn {

// device bytes a sampler of this configuration would hold, with the tensor-core plan's buffers
// where the configuration supports that schedule; -1 if the configuration is invalid
int64_t estimate_device_bytes(const bn_config &c);

// server support (bn_api.cu).  A batch whose plan is built for the given schedule kind
// (BN_SCHEDULE_AUTO: derived from the members' configured schedules, as bn_batch_create does).
int batch_create_as(bn_sampler *const *samplers, int32_t n, void *cuda_stream, int schedule,
                    bn_batch **out);
// The fastest candidate schedule for one sampler, timed on a scratch copy of its state (its
// plan, state and pass counter are left as they were); synchronises its stream.
int tune_schedule(bn_sampler *s, int32_t trial_sweeps, bn_schedule *best);
// every problem of the sampler supports the tensor-core schedule
bool tensor_capable(const bn_sampler *s);

// message returned by bn_last_error() on this thread
void set_last_error(const char *msg);

// process-wide count of kernel launches made by this library
void note_launches(long long n);
long long launch_count();

// initialisation (bn_init.cu)
cudaError_t launch_init_tables(const Problem *dprob, const Problem &h, cudaStream_t st);
cudaError_t launch_counts(const Problem *dprob, const Problem &h, cudaStream_t st);
cudaError_t launch_fetch_shifts(const Problem *dprob, const Problem &h, float *out,
                                cudaStream_t st);
cudaError_t launch_fetch_points(const Problem *dprob, const Problem &h, int pixel, float *out,
                                cudaStream_t st);
cudaError_t launch_unpack_counts(const Problem *dprob, const Problem &h, int32_t *out,
                                 cudaStream_t st);

// evaluation criterion and renderer lookup (bn_criterion.cu)
cudaError_t criterion_sums(const Problem *dprob, const Problem &h, int kind, int n_int,
                           const float *sigmas, int n_sigma, double *sums, cudaStream_t st);
cudaError_t launch_shift_table(const Problem *dprob, const Problem &h, uint32_t *out,
                               cudaStream_t st);
// error spectrum: ring of a signed frequency, the rings of a W x H tile (ring table [H][W] in DFT
// order when ring is not null; returns the ring count), and the per-ring sums of |F_t|^2 / (W H)
// over the first n_int integrands (host sums[ring count]; synchronises)
int spectrum_ring(int fx, int fy, int W, int H);
int spectrum_rings(int W, int H, std::vector<int> *ring);
cudaError_t spectrum_sums(const Problem *dprob, const Problem &h, int kind, int n_int,
                          double *sums, cudaStream_t st);
cudaError_t launch_samples(const bn_sample_table &tb, int x0, int y0, int width, int height,
                           int first, int count, int n_dims, float *out, cudaStream_t st);

// energy, Eq. 1 (bn_energy.cu)
cudaError_t launch_energy(const Problem *dprob, const Problem *hprob, int n_prob,
                          cudaStream_t st);
cudaError_t launch_energy_copy(const Problem *dprob, int n_prob, double *dev_out,
                               cudaStream_t st);

// Optional CUDA-event bracketing of kernel launches (host side).
enum KernelKind { kKEvalPlain = 0, kKResolvePlain, kKCommitPlain, kKPersistent, kKEnergy,
                  kKCounts, kKTcStencil, kKTcLists, kKTcFinalize, kKindCount };
extern const char *const kKernelNames[kKindCount];

struct KernelTimer {
    bool enabled = false;  // the evaluation kernel of every pass
    bool detail = false;   // every kernel of a pass
    struct Rec {
        int kind;
        cudaEvent_t a, b;
    };
    std::vector<Rec> pending;
    std::vector<cudaEvent_t> pool;
    long long launches[kKindCount] = {};
    double ms[kKindCount] = {};
    cudaEvent_t get();
    void begin(int kind, cudaStream_t st);
    void end(cudaStream_t st);
    cudaError_t collect();  // waits for pending events, accumulates, recycles
    void reset();
    ~KernelTimer();
};

// sweeps (bn_sweep.cu)
struct SweepLaunch {
    const Problem *dprob;   // device array of problems
    int n_prob;
    int max_M;              // largest couples-per-pass among the problems
    int count_bytes;        // 1 or 2 (all problems of one launch share it)
};
cudaError_t launch_plain_sweep(const SweepLaunch &sl, cudaStream_t st, KernelTimer *tm);
// resolve + commit of the plain schedule alone
cudaError_t launch_resolve_commit(const SweepLaunch &sl, cudaStream_t st, KernelTimer *tm);
cudaError_t launch_set_end(const Problem *dprob, int n_prob, int n_sweeps, int reset_stats,
                           cudaStream_t st);
cudaError_t launch_set_ends(const Problem *dprob, int n_prob, const int *n_sweeps_dev,
                            int reset_stats, cudaStream_t st);

// tensor-core schedule (bn_tc.cu): 8-bit counts, or 16-bit counts with N <= 512; T N^2 <= 2^27
// (centred products exact per accumulator round, class sums within int32); radius <= 8; tile
// sides >= 2 radius + 1
struct TcLaunch {
    const Problem *dprob;   // device array of problems (each with its tc_delta16 buffer)
    int n_prob;
    int max_M;
    const int4 *units;      // device [total_units] (problem, patch, x0, y0) of every 16 x 8
    int total_units;        //   patch, problem by problem
    int sms;
    const char *tmaps;      // device [n_prob] tensor maps of the count planes
    bool rounds;            // some problem needs more than one accumulator round (tc_rounds)
};
bool tc_supported(const Problem &h);
int tc_units_per_problem(const Problem &h);
// the problem's integrands are summed in more than one accumulator round (T N^2 > 2^25)
bool tc_rounds(const Problem &h);
// bytes of a problem's per-pass f16 delta rows
size_t tc_delta_bytes(const Problem &h);
// bytes of one tensor map, and its encoding for a problem's count planes (host)
int tc_tensor_map_bytes();
cudaError_t encode_tc_tensor_map(const Problem &h, void *out);
cudaError_t prepare_tc();
cudaError_t launch_tc_sweep(const TcLaunch &tl, cudaStream_t st, KernelTimer *tm);

}  // namespace bn
