// bn_sweep.cu — one pass of the parallel swap optimiser (Sec. 3.4), plain schedule:
//   k_eval_plain     candidates from the XOR-scrambled permutation; energy change of each
//                    couple on the unmodified tile; improving couples claim their two pixels
//   k_resolve_plain  an improving couple is kept unless an interacting improving couple (a
//                    pixel within the weight radius) has a higher priority
//   k_commit_plain   kept swaps move the count vectors and the shift index; pass counter += 1
// One warp per couple; count vectors are gathered straight from L2.
//
// Energy change of swapping the estimates of pixels a and b (from Eq. 1, both orders of every
// pair): with delta = k_b - k_a and S_c(p) the neighbours of p at squared distance c,
//   dL = -(4 / N^2) sum_c w_c A_c,  A_c = delta . (sum_{q in S_c(a)\b} k_q - sum_{q in S_c(b)\a} k_q)
// (the |k|^2 terms cancel because both pixels see the same number of neighbours per class).
// A_c is an exact integer; only the final weighted sum over classes is floating point.
#include "bn_launch.h"

namespace bn {
namespace {

constexpr int kPlainThreads = 256;
constexpr int kPlainWarps = kPlainThreads / 32;
constexpr int kMaxVPL = kMaxRowBytes / 16 / 32;

__device__ __forceinline__ int warp_sum(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

template <int CB>
__global__ void __launch_bounds__(kPlainThreads) k_eval_plain(const Problem *probs)
{
    const Problem &pb = probs[blockIdx.y];
    const long long s = pb.ctr[0];
    if (s >= pb.ctr[1]) return;
    __shared__ unsigned int bstat[4];
    if (threadIdx.x < 4) bstat[threadIdx.x] = 0u;
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = blockIdx.x * kPlainWarps + warp;
    if (j < pb.M) {
        const uint32_t sw = (uint32_t)s;
        const uint32_t xs = pass_xor(pb, sw);
        const int a = (int)((uint32_t)pb.perm[2 * j] ^ xs);
        const int b = (int)((uint32_t)pb.perm[2 * j + 1] ^ xs);
        float dL = 0.f, S = 0.f;
        uint8_t flags = 0;
        if (a < pb.P && b < pb.P) {
            const int nv = pb.row_bytes >> 4;
            uint4 d[kMaxVPL];
#pragma unroll
            for (int v = 0; v < kMaxVPL; ++v) {
                const int vi = v * 32 + lane;
                d[v] = vi < nv ? sub_vec<CB>(*vec_ptr(pb, b, vi), *vec_ptr(pb, a, vi))
                               : make_uint4(0u, 0u, 0u, 0u);
            }
            int A[kMaxClasses];
#pragma unroll
            for (int c = 0; c < kMaxClasses; ++c) {
                A[c] = 0;
                if (c < pb.n_cls) {
                    int acc = 0;
                    for (int side = 0; side < 2; ++side) {
                        const int p = side ? b : a, partner = side ? a : b;
                        const int px = p % pb.W, py = p / pb.W;
                        int part = 0;
                        for (int i = pb.cls_start[c]; i < pb.cls_start[c + 1]; ++i) {
                            const int q = neighbour(pb, px, py, i);
                            if (q == partner) continue;
#pragma unroll
                            for (int v = 0; v < kMaxVPL; ++v) {
                                const int vi = v * 32 + lane;
                                if (vi < nv) part = dot_vec<CB>(d[v], *vec_ptr(pb, q, vi), part);
                            }
                        }
                        acc += side ? -part : part;
                    }
                    A[c] = warp_sum(acc);
                }
            }
            couple_delta(pb, A, dL, S);
            const bool improving = (float)pb.objective * dL < 0.f;
            const bool tie = fabsf(dL) < 1e-6f * S;
            flags = kFlagValid | (improving ? kFlagImproving : 0) | (tie ? kFlagTie : 0);
            if (lane == 0) {
                atomicAdd(&bstat[kStatValid], 1u);
                if (improving) atomicAdd(&bstat[kStatImproving], 1u);
                if (tie) atomicAdd(&bstat[kStatTies], 1u);
                if (improving && pb.mode == 0) {
                    const unsigned long long key = couple_key(pb, sw, j);
                    unsigned long long *own = pb.owner + (size_t)(sw & 1u) * pb.P;
                    own[a] = key;
                    own[b] = key;
                }
            }
        }
        if (lane == 0) {
            pb.log_dE[j] = dL;
            pb.log_flags[j] = flags;
            pb.log_couples[2 * j] = a;
            pb.log_couples[2 * j + 1] = b;
        }
    }
    __syncthreads();
    if (threadIdx.x < 4 && bstat[threadIdx.x])
        atomicAdd(&pb.stats[threadIdx.x], (unsigned long long)bstat[threadIdx.x]);
}

// eight CTAs of 256 threads per SM (32 registers): more owner loads in flight, a few spills
__global__ void __launch_bounds__(kPlainThreads, 8) k_resolve_plain(const Problem *probs)
{
    const Problem &pb = probs[blockIdx.y];
    const long long s = pb.ctr[0];
    if (s >= pb.ctr[1]) return;
    __shared__ unsigned int bcommit;
    if (threadIdx.x == 0) bcommit = 0u;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = blockIdx.x * kPlainWarps + warp;
    if (j < pb.M) {
        const uint8_t flags = pb.log_flags[j];
        if (flags & kFlagImproving) {
            bool win = true;
            if (pb.mode == 0) {
                const uint32_t sw = (uint32_t)s;
                const int a = pb.log_couples[2 * j], b = pb.log_couples[2 * j + 1];
                const unsigned long long key = couple_key(pb, sw, j);
                const unsigned long long *own = pb.owner + (size_t)(sw & 1u) * pb.P;
                bool lose = false;
                for (int i = lane; i < 2 * pb.n_off; i += 32) {
                    const int side = i >= pb.n_off;
                    const int p = side ? b : a;
                    const int q = neighbour(pb, p % pb.W, p / pb.W, side ? i - pb.n_off : i);
                    if (own[q] > key) lose = true;
                }
                win = !__any_sync(0xFFFFFFFFu, lose);
            }
            if (win && lane == 0) {
                pb.log_flags[j] = flags | kFlagCommitted;
                atomicAdd(&bcommit, 1u);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && bcommit)
        atomicAdd(&pb.stats[kStatCommitted], (unsigned long long)bcommit);
}

__global__ void __launch_bounds__(kPlainThreads) k_commit_plain(const Problem *probs)
{
    const Problem &pb = probs[blockIdx.y];
    const long long s = pb.ctr[0];
    if (s >= pb.ctr[1]) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = blockIdx.x * kPlainWarps + warp;
    if (j < pb.M) {
        const uint8_t flags = pb.log_flags[j];
        const int a = pb.log_couples[2 * j], b = pb.log_couples[2 * j + 1];
        if ((flags & kFlagImproving) && pb.mode == 0 && lane == 0) {
            unsigned long long *own = pb.owner + (size_t)((uint32_t)s & 1u) * pb.P;
            own[a] = 0ull;
            own[b] = 0ull;
        }
        if (flags & kFlagCommitted) {
            for (int vi = lane; vi < (pb.row_bytes >> 4); vi += 32) {
                uint4 *ra = vec_ptr(pb, a, vi), *rb = vec_ptr(pb, b, vi);
                const uint4 t = *ra;
                *ra = *rb;
                *rb = t;
            }
            if (lane == 0) {
                const int t = pb.sidx[a];
                pb.sidx[a] = pb.sidx[b];
                pb.sidx[b] = t;
            }
        }
    }
    // the last block of this problem to finish advances the pass counter
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned long long *ticket = reinterpret_cast<unsigned long long *>(&pb.ctr[2]);
        if (atomicAdd(ticket, 1ull) == (unsigned long long)(gridDim.x - 1)) {
            *ticket = 0ull;
            pb.ctr[0] = s + 1;
            pb.stats[kStatSweeps] += 1ull;
            __threadfence();
        }
    }
}

__global__ void k_set_end(const Problem *probs, int n_sweeps, int reset_stats)
{
    const Problem &pb = probs[blockIdx.x];
    if (threadIdx.x == 0) {
        pb.ctr[1] = pb.ctr[0] + n_sweeps;
        pb.ctr[2] = 0;
    }
    if (reset_stats && threadIdx.x < kStatCount) pb.stats[threadIdx.x] = 0ull;
}

// per-problem pass budgets: ctr[1] = ctr[0] + n[i]
__global__ void k_set_ends(const Problem *probs, int n_prob, const int *n_sweeps, int reset_stats)
{
    for (int i = blockIdx.x; i < n_prob; i += gridDim.x) {
        const Problem &pb = probs[i];
        if (threadIdx.x == 0) {
            pb.ctr[1] = pb.ctr[0] + n_sweeps[i];
            pb.ctr[2] = 0;
        }
        if (reset_stats && threadIdx.x < kStatCount) pb.stats[threadIdx.x] = 0ull;
    }
}

}  // namespace

cudaError_t launch_set_ends(const Problem *dprob, int n_prob, const int *n_sweeps_dev,
                            int reset_stats, cudaStream_t st)
{
    k_set_ends<<<n_prob < 1024 ? n_prob : 1024, 32, 0, st>>>(dprob, n_prob, n_sweeps_dev,
                                                             reset_stats);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_set_end(const Problem *dprob, int n_prob, int n_sweeps, int reset_stats,
                           cudaStream_t st)
{
    k_set_end<<<n_prob, 32, 0, st>>>(dprob, n_sweeps, reset_stats);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_plain_sweep(const SweepLaunch &sl, cudaStream_t st, KernelTimer *tm)
{
    const bool timed = tm && tm->enabled;
    dim3 grid((sl.max_M + kPlainWarps - 1) / kPlainWarps, sl.n_prob);
    if (timed) tm->begin(kKEvalPlain, st);
    if (sl.count_bytes == 1)
        k_eval_plain<1><<<grid, kPlainThreads, 0, st>>>(sl.dprob);
    else
        k_eval_plain<2><<<grid, kPlainThreads, 0, st>>>(sl.dprob);
    if (timed) tm->end(st);
    const bool all = timed && tm->detail;
    if (all) tm->begin(kKResolvePlain, st);
    k_resolve_plain<<<grid, kPlainThreads, 0, st>>>(sl.dprob);
    if (all) tm->end(st);
    if (all) tm->begin(kKCommitPlain, st);
    k_commit_plain<<<grid, kPlainThreads, 0, st>>>(sl.dprob);
    if (all) tm->end(st);
    note_launches(3);
    return cudaGetLastError();
}

// the resolve and commit kernels alone (the tensor-core schedule evaluates couples itself)
cudaError_t launch_resolve_commit(const SweepLaunch &sl, cudaStream_t st, KernelTimer *tm)
{
    const bool timed = tm && tm->enabled && tm->detail;
    dim3 grid((sl.max_M + kPlainWarps - 1) / kPlainWarps, sl.n_prob);
    if (timed) tm->begin(kKResolvePlain, st);
    k_resolve_plain<<<grid, kPlainThreads, 0, st>>>(sl.dprob);
    if (timed) tm->end(st);
    if (timed) tm->begin(kKCommitPlain, st);
    k_commit_plain<<<grid, kPlainThreads, 0, st>>>(sl.dprob);
    if (timed) tm->end(st);
    note_launches(2);
    return cudaGetLastError();
}

// ---- kernel timer ---------------------------------------------------------------------------
const char *const kKernelNames[kKindCount] = {"eval_plain",       "resolve_plain",
                                               "commit_plain",     "sweep_persistent",
                                               "energy",           "counts",
                                               "stencil_tensor",   "lists_tensor",
                                               "finalize_tensor"};

cudaEvent_t KernelTimer::get()
{
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void KernelTimer::begin(int kind, cudaStream_t st)
{
    if (pending.size() >= 8192) collect();
    Rec r{kind, get(), get()};
    cudaEventRecord(r.a, st);
    pending.push_back(r);
}

void KernelTimer::end(cudaStream_t st) { cudaEventRecord(pending.back().b, st); }

cudaError_t KernelTimer::collect()
{
    cudaError_t err = cudaSuccess;
    for (auto &r : pending) {
        cudaError_t e = cudaEventSynchronize(r.b);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
        if (e == cudaSuccess) {
            launches[r.kind] += 1;
            ms[r.kind] += t;
        } else {
            err = e;
        }
        pool.push_back(r.a);
        pool.push_back(r.b);
    }
    pending.clear();
    return err;
}

void KernelTimer::reset()
{
    for (int i = 0; i < kKindCount; ++i) {
        launches[i] = 0;
        ms[i] = 0.0;
    }
}

KernelTimer::~KernelTimer()
{
    for (auto &r : pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : pool) cudaEventDestroy(e);
}

}  // namespace bn
