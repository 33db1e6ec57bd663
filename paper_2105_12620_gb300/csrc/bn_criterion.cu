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
// Spectrum (Fig. 1b): for the same error tiles, F_t = the 2-D DFT of e_t (rows, then columns,
// as direct sums with twiddle tables computed on the host in FP64), and the power |F_t|^2 / (W H)
// summed per ring of frequencies: ring = floor(rho min(W, H) + 1/2), rho the radius in cycles per
// pixel, decided in exact integer arithmetic; the mean over integrands and ring members is
// formed on the host.
//
// Layout of the scratch (per batch of B integrands): err and tmp double [P][B], integrand index
// fastest, so a warp reads B consecutive doubles of one pixel; the row transforms double2
// [H][W][B] (row y, frequency u).
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

// R[y][u][i] = sum_x e[y][x][i] tw[u x mod W], tw[k] = exp(-2 pi i k / W)
__global__ void __launch_bounds__(kCritThreads)
    k_dft_rows(int W, int H, int B, const double *err, const double2 *tw, double2 *R)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)W * H * B) return;
    const int i = (int)(idx % B);
    const int c = (int)(idx / B);  // y W + u
    const int u = c % W, y = c / W;
    const double *row = err + (size_t)y * W * B + i;
    double re = 0.0, im = 0.0;
    int k = 0;  // u x mod W
    for (int x = 0; x < W; ++x) {
        const double e = row[(size_t)x * B];
        const double2 w = tw[k];
        re = fma(e, w.x, re);
        im = fma(e, w.y, im);
        k += u;
        k -= k >= W ? W : 0;
    }
    R[idx] = make_double2(re, im);
}

// F[v][u][i] = sum_y R[y][u][i] tw[v y mod H]; |F|^2 / (W H) added to the ring of (u, v) in
// sums (per-block partial sums in shared memory first)
__global__ void __launch_bounds__(kCritThreads)
    k_dft_cols_power(int W, int H, int B, const double2 *R, const double2 *tw, const int *ring,
                     int n_rings, double *sums)
{
    extern __shared__ double sring[];  // [n_rings]
    for (int r = threadIdx.x; r < n_rings; r += blockDim.x) sring[r] = 0.0;
    __syncthreads();
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < (long long)W * H * B) {
        const int i = (int)(idx % B);
        const int c = (int)(idx / B);  // v W + u
        const int u = c % W, v = c / W;
        double re = 0.0, im = 0.0;
        int k = 0;  // v y mod H
        for (int y = 0; y < H; ++y) {
            const double2 r = R[((size_t)y * W + u) * B + i];
            const double2 w = tw[k];
            re = fma(r.x, w.x, fma(-r.y, w.y, re));
            im = fma(r.x, w.y, fma(r.y, w.x, im));
            k += v;
            k -= k >= H ? H : 0;
        }
        atomicAdd(&sring[ring[c]], (re * re + im * im) / ((double)W * (double)H));
    }
    __syncthreads();
    for (int r = threadIdx.x; r < n_rings; r += blockDim.x)
        if (sring[r] != 0.0) atomicAdd(&sums[r], sring[r]);
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

// floor(sqrt(x)) for x < 2^62
unsigned long long isqrt_u64(unsigned long long x)
{
    unsigned long long m = (unsigned long long)std::sqrt((double)x);
    while (m > 0 && m * m > x) --m;
    while ((m + 1) * (m + 1) <= x) ++m;
    return m;
}

}  // namespace

int spectrum_ring(int fx, int fy, int W, int H)
{
    // the largest b with (2b - 1) W H <= 2 L sqrt(S), S = (fx H)^2 + (fy W)^2, L = min(W, H):
    // with m = floor(2 L sqrt(S)), b = (floor(m / (W H)) + 1) / 2
    const unsigned long long L = (unsigned long long)(W < H ? W : H);
    const unsigned long long S = (unsigned long long)((long long)fx * H * fx * H) +
                                 (unsigned long long)((long long)fy * W * fy * W);
    const unsigned long long m = isqrt_u64(4ull * L * L * S);
    return (int)((m / ((unsigned long long)W * (unsigned long long)H) + 1ull) / 2ull);
}

int spectrum_rings(int W, int H, std::vector<int> *ring)
{
    int n = 0;
    if (ring) ring->assign((size_t)W * H, 0);
    for (int v = 0; v < H; ++v) {
        const int fy = 2 * v <= H ? v : v - H;
        for (int u = 0; u < W; ++u) {
            const int fx = 2 * u <= W ? u : u - W;
            const int r = spectrum_ring(fx, fy, W, H);
            if (ring) (*ring)[(size_t)v * W + u] = r;
            n = r + 1 > n ? r + 1 : n;
        }
    }
    return n;
}

cudaError_t spectrum_sums(const Problem *dprob, const Problem &h, int kind, int n_int,
                          double *sums, cudaStream_t st)
{
    const int P = h.P, W = h.W, H = h.H;
    std::vector<int> hring;
    const int n_rings = spectrum_rings(W, H, &hring);
    int B = (int)std::min<long long>(128, std::max<long long>(1, (1ll << 26) / P));
    B = std::min(B, n_int);
    std::vector<double2> hw((size_t)W + H);
    for (int k = 0; k < W; ++k)
        hw[k] = make_double2(std::cos(2.0 * M_PI * k / W), -std::sin(2.0 * M_PI * k / W));
    for (int k = 0; k < H; ++k)
        hw[(size_t)W + k] = make_double2(std::cos(2.0 * M_PI * k / H), -std::sin(2.0 * M_PI * k / H));
    double *err = nullptr, *ref = nullptr, *dsum = nullptr;
    double2 *R = nullptr, *dtw = nullptr;
    int *dring = nullptr;
    Bump *bank = nullptr;
    cudaError_t e = cudaMallocAsync(&err, sizeof(double) * (size_t)P * B, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&R, sizeof(double2) * (size_t)P * B, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&ref, sizeof(double) * B, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&bank, sizeof(Bump) * B, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&dsum, sizeof(double) * n_rings, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&dtw, sizeof(double2) * hw.size(), st);
    if (e == cudaSuccess) e = cudaMallocAsync(&dring, sizeof(int) * hring.size(), st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dtw, hw.data(), sizeof(double2) * hw.size(), cudaMemcpyHostToDevice,
                            st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dring, hring.data(), sizeof(int) * hring.size(),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dsum, 0, sizeof(double) * n_rings, st);
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
        k_dft_rows<<<grid, kCritThreads, 0, st>>>(W, H, nb, err, dtw, R);
        k_dft_cols_power<<<grid, kCritThreads, sizeof(double) * n_rings, st>>>(
            W, H, nb, R, dtw + W, dring, n_rings, dsum);
        launches += 4;
        e = cudaGetLastError();
    }
    note_launches(launches);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sums, dsum, sizeof(double) * n_rings, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    for (void *ptr : {(void *)err, (void *)R, (void *)ref, (void *)bank, (void *)dsum,
                      (void *)dtw, (void *)dring})
        if (ptr) cudaFreeAsync(ptr, st);
    const cudaError_t e2 = cudaStreamSynchronize(st);
    return e != cudaSuccess ? e : e2;
}

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
