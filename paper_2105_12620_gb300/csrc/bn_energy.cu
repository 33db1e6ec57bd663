// bn_energy.cu — Eq. 1: L = sum_p sum_{q != p, d <= r} exp(-d^2 / sigma^2) |I_p - I_q|^2.
// Exact int64 sums of |k_p - k_q|^2 per squared distance (class), then one fp32 compensated
// weighted sum per problem.
#include "bn_launch.h"

namespace bn {
namespace {

constexpr int kEnergyThreads = 256;
constexpr int kMaxVPL = kMaxRowBytes / 16 / 32;

__device__ __forceinline__ int warp_sum(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

__global__ void k_energy_clear(const Problem *probs)
{
    const Problem &pb = probs[blockIdx.x];
    if (threadIdx.x < kMaxClasses) pb.esum[threadIdx.x] = 0ull;
}

// one warp per pixel p; lanes split the count vector in 16-byte pieces
template <int CB>
__global__ void __launch_bounds__(kEnergyThreads) k_energy(const Problem *probs)
{
    const Problem &pb = probs[blockIdx.y];
    __shared__ unsigned long long bsum[kMaxClasses];
    if (threadIdx.x < kMaxClasses) bsum[threadIdx.x] = 0ull;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p = blockIdx.x * (kEnergyThreads / 32) + warp;
    if (p < pb.P) {
        const int nv = pb.row_bytes >> 4;
        const int px = p % pb.W, py = p / pb.W;
        uint4 kp[kMaxVPL];
#pragma unroll
        for (int v = 0; v < kMaxVPL; ++v) {
            const int vi = v * 32 + lane;
            kp[v] = vi < nv ? *vec_ptr(pb, p, vi) : make_uint4(0u, 0u, 0u, 0u);
        }
        for (int c = 0; c < pb.n_cls; ++c) {
            int s = 0;
            for (int i = pb.cls_start[c]; i < pb.cls_start[c + 1]; ++i) {
                const int q = neighbour(pb, px, py, i);
#pragma unroll
                for (int v = 0; v < kMaxVPL; ++v) {
                    const int vi = v * 32 + lane;
                    if (vi < nv) {
                        const uint4 k = *vec_ptr(pb, q, vi);
                        s = sqdiff_word<CB>(kp[v].x, k.x, s);
                        s = sqdiff_word<CB>(kp[v].y, k.y, s);
                        s = sqdiff_word<CB>(kp[v].z, k.z, s);
                        s = sqdiff_word<CB>(kp[v].w, k.w, s);
                    }
                }
            }
            s = warp_sum(s);
            if (lane == 0 && s) atomicAdd(&bsum[c], (unsigned long long)(long long)s);
        }
    }
    __syncthreads();
    if (threadIdx.x < pb.n_cls && bsum[threadIdx.x])
        atomicAdd(&pb.esum[threadIdx.x], bsum[threadIdx.x]);
}

__global__ void k_energy_finalize(const Problem *probs)
{
    const Problem &pb = probs[blockIdx.x];
    if (threadIdx.x != 0) return;
    F2 acc = {0.f, 0.f};
    for (int c = 0; c < pb.n_cls; ++c) add_weighted_i64(acc, pb.w[c], (long long)pb.esum[c]);
    renorm(acc);
    // 1 / N^2 is a power of two: exact scaling of both parts
    const double inv = 1.0 / ((double)pb.N * (double)pb.N);
    *pb.energy_out = ((double)acc.hi + (double)acc.lo) * inv;
}

}  // namespace

cudaError_t launch_energy(const Problem *dprob, const Problem *hprob, int n_prob,
                          cudaStream_t st)
{
    int maxP = 0, cb = hprob[0].count_bytes;
    for (int i = 0; i < n_prob; ++i) maxP = hprob[i].P > maxP ? hprob[i].P : maxP;
    k_energy_clear<<<n_prob, 32, 0, st>>>(dprob);
    dim3 grid((maxP + kEnergyThreads / 32 - 1) / (kEnergyThreads / 32), n_prob);
    if (cb == 1)
        k_energy<1><<<grid, kEnergyThreads, 0, st>>>(dprob);
    else
        k_energy<2><<<grid, kEnergyThreads, 0, st>>>(dprob);
    k_energy_finalize<<<n_prob, 32, 0, st>>>(dprob);
    note_launches(3);
    return cudaGetLastError();
}

namespace {
__global__ void k_energy_copy(const Problem *probs, double *out)
{
    out[blockIdx.x] = *probs[blockIdx.x].energy_out;
}
}  // namespace

cudaError_t launch_energy_copy(const Problem *dprob, int n_prob, double *dev_out,
                               cudaStream_t st)
{
    k_energy_copy<<<n_prob, 1, 0, st>>>(dprob, dev_out);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace bn
