// bn_noalloc.cu — Eq. 1 evaluated without any device allocation.
//
// Some callers cannot allocate device memory: code that runs inside another framework's
// memory pool or arena (where a stray cudaMalloc would bypass its accounting or trigger a
// device-wide synchronisation), real-time loops that must not stall on the allocator, and
// plug-ins that are only handed pre-allocated buffers.  bn_evaluate_energy_noalloc serves
// them: the caller passes the count fields and the output buffer, and the only scratch (the
// per-class integer sums) lives in the fixed file-scope array below, which every GPU that loads
// this library holds until the process exits.
//
// The array is shared by all calls: each call clears the part it uses before accumulating, so
// a call sees nothing of the previous one, but two calls whose work overlaps on the GPU (on
// different streams, or on the same device from different threads without ordering) race on it
// and may return wrong energies.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "bn_launch.h"
#include "bn_sampler.h"

namespace bn {
namespace {

constexpr int kNoAllocMaxFields = 64;  // count fields per call
constexpr int kNoAllocThreads = 256;

// Per-field, per-class sums of |k_p - k_q|^2 (two's complement int64): 64 x 32 x 8 B = 16 KiB.
static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNoAllocMaxFields * kMaxClasses];

constexpr int kMaxDevices = 64;
std::atomic<void *> g_scratch_ptr[kMaxDevices] = {};  // device address of the array, per device

struct Stencil {
    int n_off, n_cls;
    float w[kMaxClasses];
    int cls_start[kMaxClasses + 1];
    int off[kMaxOffsets];  // (dx & 0xFFFF) | (dy << 16)
};

__global__ void k_noalloc_clear(unsigned long long *scratch, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) scratch[i] = 0ull;
}

// one warp per pixel of one field (blockIdx.y); counts are int32 [P][T] row-major per field
__global__ void __launch_bounds__(kNoAllocThreads)
    k_noalloc_energy(const int32_t *counts, int W, int H, int T, Stencil st,
                     unsigned long long *scratch)
{
    __shared__ unsigned long long bsum[kMaxClasses];
    if (threadIdx.x < kMaxClasses) bsum[threadIdx.x] = 0ull;
    __syncthreads();
    const int P = W * H;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p = blockIdx.x * (kNoAllocThreads / 32) + warp;
    const int32_t *field = counts + (size_t)blockIdx.y * P * T;
    if (p < P) {
        const int px = p % W, py = p / W;
        const int32_t *kp = field + (size_t)p * T;
        for (int c = 0; c < st.n_cls; ++c) {
            long long s = 0;
            for (int i = st.cls_start[c]; i < st.cls_start[c + 1]; ++i) {
                const int o = st.off[i];
                const int dx = (int)(int16_t)(o & 0xFFFF), dy = o >> 16;
                int qx = px + dx, qy = py + dy;
                qx += qx < 0 ? W : 0;
                qx -= qx >= W ? W : 0;
                qy += qy < 0 ? H : 0;
                qy -= qy >= H ? H : 0;
                const int32_t *kq = field + ((size_t)qy * W + qx) * T;
                for (int t = lane; t < T; t += 32) {
                    const long long d = (long long)kp[t] - kq[t];
                    s += d * d;
                }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, off);
            if (lane == 0 && s) atomicAdd(&bsum[c], (unsigned long long)s);
        }
    }
    __syncthreads();
    if (threadIdx.x < st.n_cls && bsum[threadIdx.x])
        atomicAdd(&scratch[blockIdx.y * kMaxClasses + threadIdx.x], bsum[threadIdx.x]);
}

// E = (1 / N^2) sum_c w_c S_c, fp32 compensated, one thread per field
__global__ void k_noalloc_finalize(const unsigned long long *scratch, int n_fields, int N,
                                   Stencil st, double *energy)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n_fields) return;
    F2 acc = {0.f, 0.f};
    for (int c = 0; c < st.n_cls; ++c)
        add_weighted_i64(acc, st.w[c], (long long)scratch[f * kMaxClasses + c]);
    renorm(acc);
    const double inv = 1.0 / ((double)N * (double)N);
    energy[f] = ((double)acc.hi + (double)acc.lo) * inv;
}

int nfail(int code, const std::string &msg)
{
    set_last_error(msg.c_str());
    return code;
}

bool canonical(int d, int n)
{
    const int o = ((d % n) + n) % n;
    const int rep = (2 * o <= n) ? o : o - n;
    return rep == d;
}

}  // namespace
}  // namespace bn

// Eq. 1 of every field, with no device allocation (see the header for the contract).
extern "C" int bn_evaluate_energy_noalloc(const int32_t *counts, int32_t n_fields, int32_t width,
                                          int32_t height, int32_t n_points, int32_t n_integrands,
                                          float sigma, int32_t radius, double *energy,
                                          void *cuda_stream)
{
    using namespace bn;
    if (!counts || !energy) return nfail(BN_ERR_INVALID_ARG, "null counts or energy pointer");
    if (n_fields < 1 || n_fields > kNoAllocMaxFields)
        return nfail(BN_ERR_INVALID_ARG, "n_fields must be in [1, " +
                                             std::to_string(kNoAllocMaxFields) +
                                             "]: the fixed scratch array holds that many fields");
    if (width < 2 || height < 2 || (long long)width * height > (1ll << 22))
        return nfail(BN_ERR_INVALID_ARG, "width, height >= 2 and width*height <= 2^22");
    if (n_points < 2 || n_points > 1024 || (n_points & (n_points - 1)))
        return nfail(BN_ERR_INVALID_ARG, "n_points must be a power of two in [2, 1024]");
    if (n_integrands < 1 || n_integrands > 4096)
        return nfail(BN_ERR_INVALID_ARG, "n_integrands must be in [1, 4096]");
    if (!(sigma > 0.f) || !std::isfinite(sigma))
        return nfail(BN_ERR_INVALID_ARG, "sigma must be positive");
    if (radius < 1 || radius > 8) return nfail(BN_ERR_INVALID_ARG, "radius must be in [1, 8]");

    // stencil of distinct torus neighbours within the radius, grouped by squared distance
    Stencil st;
    memset(&st, 0, sizeof st);
    int n = 0;
    for (int d2 = 1; d2 <= radius * radius; ++d2) {
        const int first = n;
        for (int dy = -radius; dy <= radius; ++dy)
            for (int dx = -radius; dx <= radius; ++dx)
                if (dx * dx + dy * dy == d2 && canonical(dx, width) && canonical(dy, height))
                    st.off[n++] = (dx & 0xFFFF) | (dy << 16);
        if (n > first) {
            st.cls_start[st.n_cls] = first;
            st.w[st.n_cls] = (float)std::exp(-(double)d2 / ((double)sigma * sigma));
            ++st.n_cls;
        }
    }
    st.n_off = n;
    st.cls_start[st.n_cls] = n;

    // set-up, once per device, with that device current: the device address of the array
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return nfail(BN_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return nfail(BN_ERR_CUDA, "device index out of range");
    if (!g_scratch_ptr[dev].load()) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr)
            return nfail(BN_ERR_CUDA, std::string("cudaGetSymbolAddress of the scratch array: ") +
                                          cudaGetErrorString(e));
        g_scratch_ptr[dev].store(ptr);
    }
    auto *scratch = static_cast<unsigned long long *>(g_scratch_ptr[dev].load());
    cudaStream_t stream = (cudaStream_t)cuda_stream;

    // an error the caller left pending is reported as such (and left pending), not taken for
    // a failure of the launches below
    e = cudaPeekAtLastError();
    if (e != cudaSuccess)
        return nfail(BN_ERR_CUDA, std::string("a CUDA error was pending before the call: ") +
                                      cudaGetErrorString(e));
    const int used = n_fields * kMaxClasses;
    k_noalloc_clear<<<(used + 255) / 256, 256, 0, stream>>>(scratch, used);
    e = cudaGetLastError();
    if (e != cudaSuccess) return nfail(BN_ERR_CUDA, std::string("launch of the clear: ") + cudaGetErrorString(e));
    const int P = width * height;
    dim3 grid((P + kNoAllocThreads / 32 - 1) / (kNoAllocThreads / 32), n_fields);
    k_noalloc_energy<<<grid, kNoAllocThreads, 0, stream>>>(counts, width, height, n_integrands,
                                                           st, scratch);
    e = cudaGetLastError();
    if (e != cudaSuccess) return nfail(BN_ERR_CUDA, std::string("launch of the class sums: ") + cudaGetErrorString(e));
    k_noalloc_finalize<<<(n_fields + 63) / 64, 64, 0, stream>>>(scratch, n_fields, n_points, st,
                                                                energy);
    note_launches(3);
    e = cudaGetLastError();
    if (e != cudaSuccess) return nfail(BN_ERR_CUDA, std::string("launch of the weighted sum: ") + cudaGetErrorString(e));
    return BN_OK;
}
