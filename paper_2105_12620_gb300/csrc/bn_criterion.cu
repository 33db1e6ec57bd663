// bn_criterion.cu — evaluation of a sampler tile (Sec. 3.3, Sec. 3.5) and the renderer lookup
// (Sec. 3.1, Sec. 3.2).
//
// Criterion: for each integrand t, the error tile e_t(p) = I_p - I_ref (estimate minus exact
// integral) is filtered by the wrapped, sampled Gaussian of standard deviation sigma (separable,
// periodic on the tile, weights normalised to 1) and the RMSE over integrands and pixels is
// reported per sigma.  Integrands: the sampler's own Heavisides (estimate k_p[t] / N, reference
// the exact area of the half-plane within the unit square) or smooth Gaussian bumps drawn from
// Philox tag 7 (estimate: mean over the pixel's N shifted lattice points, reference: product of
// erf differences).  Everything is FP64: the filtered errors at wide sigma are small differences
// of much larger terms.
//
// Layout of the scratch (per batch of B integrands): err and tmp double [P][B], integrand index
// fastest, so a warp reads B consecutive doubles of one pixel.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "bn_device.cuh"
#include "bn_launch.h"
#include "bn_sample.cuh"

namespace bn {
namespace {

constexpr uint32_t kTagBump = 7u;
constexpr int kCritThreads = 256;

// area of {a x + b y < c} within [0,1]^2: clip the square's polygon by the half-plane and take
// the shoelace area of the rest
__device__ double half_plane_area(double a, double b, double c)
{
    const double sx[4] = {0.0, 1.0, 1.0, 0.0}, sy[4] = {0.0, 0.0, 1.0, 1.0};
    double ox[8], oy[8];
    int n = 0;
    for (int i = 0; i < 4; ++i) {
        const int j = (i + 1) & 3;
        const double fi = a * sx[i] + b * sy[i] - c, fj = a * sx[j] + b * sy[j] - c;
        if (fi < 0.0) {
            ox[n] = sx[i];
            oy[n] = sy[i];
            ++n;
        }
        if ((fi < 0.0) != (fj < 0.0)) {
            const double t = fi / (fi - fj);
            ox[n] = sx[i] + t * (sx[j] - sx[i]);
            oy[n] = sy[i] + t * (sy[j] - sy[i]);
            ++n;
        }
    }
    double area = 0.0;
    for (int i = 0; i < n; ++i) {
        const int j = (i + 1) % n;
        area += ox[i] * oy[j] - ox[j] * oy[i];
    }
    return n < 3 ? 0.0 : fabs(area) * 0.5;
}

// reference integral of integrand t (first + i of the bank) into ref[i]
__global__ void k_heaviside_refs(const Problem *probs, int first, int n, double *ref)
{
    const Problem &pb = *probs;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int t = first + i;
    ref[i] = half_plane_area((double)pb.ha[t], (double)pb.hb[t], (double)pb.hC[t] * 0x1p-24);
}

struct Bump {
    double cx, cy, inv2s2, ref;
};

__global__ void k_bump_bank(const Problem *probs, int first, int n, Bump *bank)
{
    const Problem &pb = *probs;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 w = draw(pb, (uint32_t)(first + i), 0u, kTagBump);
    const double cx = (double)w.x * 0x1p-32, cy = (double)w.y * 0x1p-32;
    const double s = 0.05 + 0.45 * ((double)w.z * 0x1p-32);
    const double r = s * 1.4142135623730951;      // s sqrt(2)
    const double k = s * 1.2533141373155003;      // s sqrt(pi / 2)
    const double ix = k * (erf((1.0 - cx) / r) + erf(cx / r));
    const double iy = k * (erf((1.0 - cy) / r) + erf(cy / r));
    bank[i] = Bump{cx, cy, 1.0 / (2.0 * s * s), ix * iy};
}

// e[p][i] = k_p[first + i] / N - ref[i]
template <typename CT>
__global__ void k_err_heaviside(const Problem *probs, int first, int B, const double *ref,
                                double *err)
{
    const Problem &pb = *probs;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)pb.P * B) return;
    const int p = (int)(idx / B), i = (int)(idx % B);
    const int byte = (first + i) * (int)sizeof(CT);
    const CT k = reinterpret_cast<const CT *>(chunk_ptr(pb, p, byte >> 7))[(byte & 127) /
                                                                          (int)sizeof(CT)];
    err[idx] = (double)k * (1.0 / (double)pb.N) - ref[i];  // N = 2^m: exact, no division
}

// e[p][i] = (1/N) sum_k f_i(s_p^k) - ref_i for the bumps; one warp per pixel, lanes over bumps
__global__ void k_err_bumps(const Problem *probs, int B, const Bump *bank, double *err)
{
    const Problem &pb = *probs;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= pb.P) return;
    const int p = warp, src = pb.sidx[p];
    const uint32_t ux = pb.U[2 * src], uy = pb.U[2 * src + 1];
    const int m = pb.m;
    for (int i = lane; i < B; i += 32) {
        const Bump bp = bank[i];
        double acc = 0.0;
        for (int k = 0; k < pb.N; ++k) {
            const uint32_t rk = __brev((uint32_t)k) >> (32 - m);
            const uint32_t sx = rk << (32 - m);
            const uint32_t sy = ((rk * (uint32_t)pb.g) & (uint32_t)(pb.N - 1)) << (32 - m);
            const double x = (double)(sx + ux) * 0x1p-32, y = (double)(sy + uy) * 0x1p-32;
            const double dx = x - bp.cx, dy = y - bp.cy;
            acc += exp(-(dx * dx + dy * dy) * bp.inv2s2);
        }
        err[(size_t)p * B + i] = acc * (1.0 / (double)pb.N) - bp.ref;
    }
}

// out[y][x][i] = sum_j w_j in[y][(x + o_j) mod W][i]   (dir 0)
// out[y][x][i] = sum_j w_j in[(y + o_j) mod H][x][i]   (dir 1), and the squares summed
template <bool VERTICAL>
__global__ void __launch_bounds__(kCritThreads)
    k_blur(int W, int H, int B, const double *in, double *out, const int *off, const double *w,
           int n_taps, double *sq_sum)
{
    __shared__ double red[kCritThreads / 32];
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)W * H * B;
    double v = 0.0;
    if (idx < total) {
        const int i = (int)(idx % B);
        const int p = (int)(idx / B);
        const int x = p % W, y = p / W;
        for (int j = 0; j < n_taps; ++j) {
            int q;
            if (VERTICAL) {
                int yy = y + off[j];
                yy -= yy >= H ? H : 0;
                q = yy * W + x;
            } else {
                int xx = x + off[j];
                xx -= xx >= W ? W : 0;
                q = y * W + xx;
            }
            v += w[j] * in[(size_t)q * B + i];
        }
        if (!VERTICAL) out[idx] = v;
    }
    if (VERTICAL) {
        double s = v * v;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int k = 0; k < kCritThreads / 32; ++k) t += red[k];
            atomicAdd(sq_sum, t);
        }
    }
}

// renderer lookup into out[r][i][j][d] for screen pixels (x0 + i, y0 + r), samples first + j
__global__ void k_samples(bn_sample_table tb, int x0, int y0, int width, int height, int first,
                          int count, int n_dims, float *out)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)width * height * count) return;
    const int j = (int)(idx % count);
    const long long pix = idx / count;
    const int i = (int)(pix % width), r = (int)(pix / width);
    for (int d = 0; d < n_dims; ++d)
        out[idx * n_dims + d] = bn_sample(tb, x0 + i, y0 + r, first + j, d);
}

__global__ void k_shift_table(const Problem *probs, uint32_t *out)
{
    const Problem &pb = *probs;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= pb.P) return;
    const int src = pb.sidx[p];
    out[2 * p] = pb.U[2 * src];
    out[2 * p + 1] = pb.U[2 * src + 1];
}

// taps of the wrapped sampled Gaussian along a tile side of n pixels (offsets in [0, n))
void gaussian_taps(int n, double sigma, std::vector<int> &off, std::vector<double> &w)
{
    off.clear();
    w.clear();
    if (!(sigma > 0.0)) {
        off.push_back(0);
        w.push_back(1.0);
        return;
    }
    std::vector<double> full(n, 0.0);
    const long long reach = (long long)std::ceil(12.0 * sigma) + n;
    for (int d = 0; d < n; ++d) {
        double s = 0.0;
        for (long long x = d - ((reach / n) + 1) * (long long)n; x <= reach; x += n)
            s += std::exp(-(double)(x * x) / (2.0 * sigma * sigma));
        full[d] = s;
    }
    double total = 0.0, peak = 0.0;
    for (double v : full) {
        total += v;
        peak = v > peak ? v : peak;
    }
    for (int d = 0; d < n; ++d)
        if (full[d] > 1e-20 * peak) {
            off.push_back(d);
            w.push_back(full[d] / total);
        }
}

}  // namespace

cudaError_t criterion_sums(const Problem *dprob, const Problem &h, int kind, int n_int,
                           const float *sigmas, int n_sigma, double *sums, cudaStream_t st)
{
    const int P = h.P;
    int B = (int)std::min<long long>(128, std::max<long long>(1, (1ll << 27) / P));
    B = std::min(B, n_int);
    double *err = nullptr, *tmp = nullptr, *ref = nullptr, *dsum = nullptr, *dw = nullptr;
    int *doff = nullptr;
    Bump *bank = nullptr;
    const int max_taps = std::max(h.W, h.H);
    std::vector<std::vector<int>> ox(n_sigma), oy(n_sigma);
    std::vector<std::vector<double>> wx(n_sigma), wy(n_sigma);
    for (int s = 0; s < n_sigma; ++s) {
        gaussian_taps(h.W, sigmas[s], ox[s], wx[s]);
        gaussian_taps(h.H, sigmas[s], oy[s], wy[s]);
    }
    cudaError_t e = cudaMallocAsync(&err, sizeof(double) * (size_t)P * B, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&tmp, sizeof(double) * (size_t)P * B, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&ref, sizeof(double) * B, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&bank, sizeof(Bump) * B, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&dsum, sizeof(double) * n_sigma, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&doff, sizeof(int) * 2 * n_sigma * max_taps, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&dw, sizeof(double) * 2 * n_sigma * max_taps, st);
    // taps of every sigma, x then y, at fixed strides
    std::vector<int> hoff((size_t)2 * n_sigma * max_taps, 0);
    std::vector<double> hw((size_t)2 * n_sigma * max_taps, 0.0);
    for (int s = 0; s < n_sigma; ++s) {
        std::copy(ox[s].begin(), ox[s].end(), hoff.begin() + (size_t)(2 * s) * max_taps);
        std::copy(wx[s].begin(), wx[s].end(), hw.begin() + (size_t)(2 * s) * max_taps);
        std::copy(oy[s].begin(), oy[s].end(), hoff.begin() + (size_t)(2 * s + 1) * max_taps);
        std::copy(wy[s].begin(), wy[s].end(), hw.begin() + (size_t)(2 * s + 1) * max_taps);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(doff, hoff.data(), sizeof(int) * hoff.size(), cudaMemcpyHostToDevice,
                            st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dw, hw.data(), sizeof(double) * hw.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dsum, 0, sizeof(double) * n_sigma, st);
    int launches = 0;
    for (int first = 0; e == cudaSuccess && first < n_int; first += B) {
        const int nb = std::min(B, n_int - first);
        const long long cells = (long long)P * nb;
        const int grid = (int)((cells + kCritThreads - 1) / kCritThreads);
        if (kind == BN_INTEGRANDS_HEAVISIDE) {
            k_heaviside_refs<<<(nb + 127) / 128, 128, 0, st>>>(dprob, first, nb, ref);
            if (h.count_bytes == 1)
                k_err_heaviside<uint8_t><<<grid, kCritThreads, 0, st>>>(dprob, first, nb, ref, err);
            else
                k_err_heaviside<uint16_t><<<grid, kCritThreads, 0, st>>>(dprob, first, nb, ref,
                                                                         err);
        } else {
            k_bump_bank<<<(nb + 127) / 128, 128, 0, st>>>(dprob, first, nb, bank);
            k_err_bumps<<<(P * 32 + kCritThreads - 1) / kCritThreads, kCritThreads, 0, st>>>(
                dprob, nb, bank, err);
        }
        launches += 2;
        for (int s = 0; s < n_sigma; ++s) {
            const int *ofx = doff + (size_t)(2 * s) * max_taps;
            const int *ofy = doff + (size_t)(2 * s + 1) * max_taps;
            const double *w_x = dw + (size_t)(2 * s) * max_taps;
            const double *w_y = dw + (size_t)(2 * s + 1) * max_taps;
            k_blur<false><<<grid, kCritThreads, 0, st>>>(h.W, h.H, nb, err, tmp, ofx, w_x,
                                                         (int)ox[s].size(), nullptr);
            k_blur<true><<<grid, kCritThreads, 0, st>>>(h.W, h.H, nb, tmp, nullptr, ofy, w_y,
                                                        (int)oy[s].size(), dsum + s);
            launches += 2;
        }
        e = cudaGetLastError();
    }
    note_launches(launches);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sums, dsum, sizeof(double) * n_sigma, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    for (void *ptr : {(void *)err, (void *)tmp, (void *)ref, (void *)bank, (void *)dsum,
                      (void *)doff, (void *)dw})
        if (ptr) cudaFreeAsync(ptr, st);
    const cudaError_t e2 = cudaStreamSynchronize(st);
    return e != cudaSuccess ? e : e2;
}

cudaError_t launch_shift_table(const Problem *dprob, const Problem &h, uint32_t *out,
                               cudaStream_t st)
{
    k_shift_table<<<(h.P + 255) / 256, 256, 0, st>>>(dprob, out);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_samples(const bn_sample_table &tb, int x0, int y0, int width, int height,
                           int first, int count, int n_dims, float *out, cudaStream_t st)
{
    const long long n = (long long)width * height * count;
    k_samples<<<(int)((n + 255) / 256), 256, 0, st>>>(tb, x0, y0, width, height, first, count,
                                                      n_dims, out);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace bn
