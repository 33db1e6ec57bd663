// bn_init.cu — initialisation kernels: shifts, Heaviside bank, candidate permutation and the
// counting kernel (test-integrand estimates of every pixel), plus fetch helpers.
#include <atomic>

#include "bn_launch.h"

namespace bn {
namespace {

// Tile of scrambling parameters (Sec. 2): u_p uniform in [0,1)^2, 24 significant bits.
__global__ void k_init_shifts(const Problem *probs)
{
    const Problem &pb = *probs;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= pb.P) return;
    const uint4 r = draw(pb, (uint32_t)p, 0u, kTagShift);
    pb.U[2 * p] = r.x & 0xFFFFFF00u;
    pb.U[2 * p + 1] = r.y & 0xFFFFFF00u;
    pb.sidx[p] = p;
}

// Randomly oriented Heavisides (Sec. 2, Fig. 1b): integer normal uniform in the disc of radius
// 2^15, offset uniform over the projection of the unit square on the normal.
__global__ void k_init_bank(const Problem *probs)
{
    const Problem &pb = *probs;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= pb.T) return;
    int a = 1, b = 0;
    uint32_t roff = 0x80000000u;
    for (uint32_t attempt = 0; attempt < 64u; ++attempt) {
        const uint4 r = draw(pb, (uint32_t)t, attempt, kTagHeavi);
        const int ca = (int)(r.x >> 16) - 32768, cb = (int)(r.y >> 16) - 32768;
        const long long q = (long long)ca * ca + (long long)cb * cb;
        if (q > 0 && q <= (1ll << 30)) {
            a = ca;
            b = cb;
            roff = r.z;
            break;
        }
    }
    const long long lo = (long long)min(a, 0) + min(b, 0);
    const long long hi = (long long)max(a, 0) + max(b, 0);
    pb.ha[t] = a;
    pb.hb[t] = b;
    pb.hC[t] = lo * (1ll << 24) + (long long)(((unsigned long long)roff *
                                               (unsigned long long)(hi - lo)) >> 8);
}

// Candidate permutation (Sec. 3.4) as a swap-or-not shuffle (Hoang, Morris, Rogaway 2012) of
// [0, 2^L); also its inverse, so that a pixel can find its own candidate slot.
__global__ void k_init_perm(const Problem *probs, int rounds)
{
    const Problem &pb = *probs;
    const uint32_t n = 1u << pb.L, mask = n - 1u;
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t x = i;
    for (int r = 0; r < rounds; ++r) {
        const uint32_t K = draw(pb, (uint32_t)r, 0u, kTagPermKey).x & mask;
        const uint32_t partner = x ^ K;
        const uint32_t hi = x > partner ? x : partner;
        if (draw(pb, hi, (uint32_t)r, kTagPermBit).x & 1u) x = partner;
    }
    pb.perm[i] = (int32_t)x;
    pb.perm_inv[x] = (int32_t)i;
}

__global__ void k_clear_state(const Problem *probs)
{
    const Problem &pb = *probs;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 2 * pb.P) pb.owner[i] = 0ull;
    if (i < kStatCount) pb.stats[i] = 0ull;
    if (i < 4) pb.ctr[i] = 0;
    if (i < pb.tc_npx * pb.tc_npy) pb.tc_cnt[i] = 0;
}

// Counting kernel (Sec. 2 and Sec. 3.2): k_p[t] = #{k < N : a_t X + b_t Y < C_t} with
// (X, Y) = ((S(k) + U_p) mod 2^32) >> 8, S(k) = (rev_m(k), rev_m(k) g mod N) * 2^(32-m).
// One thread per integrand t, PPB pixels per block; lattice in shared memory.
constexpr int kCountThreads = 256;
constexpr int kCountPixels = 8;

template <typename CT>
__global__ void __launch_bounds__(kCountThreads) k_counts(const Problem *probs)
{
    const Problem &pb = *probs;
    extern __shared__ uint32_t lat[];  // [2][N]
    const int N = pb.N, m = pb.m;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const uint32_t rk = __brev((uint32_t)k) >> (32 - m);
        lat[k] = rk << (32 - m);
        lat[N + k] = ((rk * (uint32_t)pb.g) & (uint32_t)(N - 1)) << (32 - m);
    }
    __syncthreads();
    const int t = blockIdx.y * blockDim.x + threadIdx.x;
    const int row_elems = pb.row_bytes / (int)sizeof(CT);
    if (t >= row_elems) return;
    const bool real = t < pb.T;
    const long long a = real ? pb.ha[t] : 0, b = real ? pb.hb[t] : 0;
    const long long C = real ? pb.hC[t] : 0;
    const int p0 = blockIdx.x * kCountPixels;
    const int p1 = min(p0 + kCountPixels, pb.P);
    for (int p = p0; p < p1; ++p) {
        const int src = pb.sidx[p];
        const uint32_t ux = pb.U[2 * src], uy = pb.U[2 * src + 1];
        int cnt = 0;
        if (real) {
            for (int k = 0; k < N; ++k) {
                const uint32_t X = (lat[k] + ux) >> 8, Y = (lat[N + k] + uy) >> 8;
                cnt += (a * (long long)X + b * (long long)Y < C) ? 1 : 0;
            }
        }
        const int byte = t * (int)sizeof(CT);
        reinterpret_cast<CT *>(chunk_ptr(pb, p, byte >> 7))[(byte & 127) / (int)sizeof(CT)] =
            (CT)cnt;
    }
}

__global__ void k_fetch_shifts(const Problem *probs, float *out)
{
    const Problem &pb = *probs;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= pb.P) return;
    const int src = pb.sidx[p];
    out[2 * p] = (float)pb.U[2 * src] * 2.3283064365386963e-10f;  // 2^-32, exact
    out[2 * p + 1] = (float)pb.U[2 * src + 1] * 2.3283064365386963e-10f;
}

__global__ void k_fetch_points(const Problem *probs, int pixel, float *out)
{
    const Problem &pb = *probs;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= pb.N) return;
    const int m = pb.m, src = pb.sidx[pixel];
    const uint32_t rk = __brev((uint32_t)k) >> (32 - m);
    const uint32_t sx = rk << (32 - m), sy = ((rk * (uint32_t)pb.g) & (uint32_t)(pb.N - 1))
                                                 << (32 - m);
    out[2 * k] = (float)(sx + pb.U[2 * src]) * 2.3283064365386963e-10f;
    out[2 * k + 1] = (float)(sy + pb.U[2 * src + 1]) * 2.3283064365386963e-10f;
}

template <typename CT>
__global__ void k_unpack_counts(const Problem *probs, int32_t *out)
{
    const Problem &pb = *probs;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)pb.P * pb.T) return;
    const int p = (int)(i / pb.T), t = (int)(i % pb.T);
    const int byte = t * (int)sizeof(CT);
    out[i] = reinterpret_cast<const CT *>(chunk_ptr(pb, p, byte >> 7))[(byte & 127) /
                                                                      (int)sizeof(CT)];
}

int perm_rounds(int L) { return 6 * L < 12 ? 12 : 6 * L; }

std::atomic<long long> g_launches{0};

}  // namespace

void note_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

cudaError_t launch_init_tables(const Problem *dprob, const Problem &h, cudaStream_t st)
{
    const int nt = 256;
    k_init_shifts<<<(h.P + nt - 1) / nt, nt, 0, st>>>(dprob);
    k_init_bank<<<(h.T + nt - 1) / nt, nt, 0, st>>>(dprob);
    k_init_perm<<<((1 << h.L) + nt - 1) / nt, nt, 0, st>>>(dprob, perm_rounds(h.L));
    const int nclear = 2 * h.P > h.M ? 2 * h.P : h.M;
    k_clear_state<<<(nclear + nt - 1) / nt, nt, 0, st>>>(dprob);
    note_launches(4);
    return cudaGetLastError();
}

cudaError_t launch_counts(const Problem *dprob, const Problem &h, cudaStream_t st)
{
    const int row_elems = h.row_bytes / h.count_bytes;
    dim3 grid((h.P + kCountPixels - 1) / kCountPixels, (row_elems + kCountThreads - 1) /
                                                           kCountThreads);
    const size_t smem = sizeof(uint32_t) * 2 * h.N;
    if (h.count_bytes == 1)
        k_counts<uint8_t><<<grid, kCountThreads, smem, st>>>(dprob);
    else
        k_counts<uint16_t><<<grid, kCountThreads, smem, st>>>(dprob);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_fetch_shifts(const Problem *dprob, const Problem &h, float *out,
                                cudaStream_t st)
{
    k_fetch_shifts<<<(h.P + 255) / 256, 256, 0, st>>>(dprob, out);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_fetch_points(const Problem *dprob, const Problem &h, int pixel, float *out,
                                cudaStream_t st)
{
    k_fetch_points<<<(h.N + 255) / 256, 256, 0, st>>>(dprob, pixel, out);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_unpack_counts(const Problem *dprob, const Problem &h, int32_t *out,
                                 cudaStream_t st)
{
    const long long n = (long long)h.P * h.T;
    const int blocks = (int)((n + 255) / 256);
    if (h.count_bytes == 1)
        k_unpack_counts<uint8_t><<<blocks, 256, 0, st>>>(dprob, out);
    else
        k_unpack_counts<uint16_t><<<blocks, 256, 0, st>>>(dprob, out);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace bn
