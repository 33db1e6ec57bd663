// bn_persistent.cu — the parallel swap optimiser (Sec. 3.4) as one cooperative, persistent
// launch that runs many passes over a batch of problems (tiles x pairs of dimensions).
//
// Per pass, two phases separated by grid barriers:
//   phase 1 (evaluate): the work unit is a block of BX x BY pixels of one problem and a range of
//     128-byte chunks of the count vectors.  The CTA finds the block's proposed pixels (pixels
//     that belong to a valid couple of this pass), stages the block's window (block plus a halo
//     of the weight radius, wrapped on the torus) chunk by chunk into shared memory with
//     cp.async double buffering, together with each proposed pixel's partner chunk, and every
//     warp accumulates, for its proposed pixels, the exact integer sums
//         A_c(p) += delta_p . k_q,   q in S_c(p),   delta_p = k_partner - k_p
//     with the 112 stencil offsets as compile-time shared-memory displacements (one IDP4A per
//     4 counts).  The contribution of the partner itself (when it lies in the neighbourhood) is
//     removed afterwards.  Each side's class sums go to global memory; the last of the
//     2 x tsplit contributions of a couple computes dL in fp32 (compensated), sets the flags,
//     logs, and, if the swap improves the objective, claims the couple's two pixels in the
//     owner grid of this pass's parity.
//   phase 2 (resolve + commit): one warp per couple: an improving couple is kept unless an
//     interacting improving couple (a pixel within the radius) has a higher priority; kept
//     swaps move the count vectors and the shift index.  Owner entries of the previous pass are
//     cleared here.
// Data written inside the launch is read back with L2-only loads (.cg) because L1 is not
// coherent across SMs.  Grid barriers spin with a clock budget; on timeout the kernel records
// an error and every block returns.
#include <utility>

#include "bn_launch.h"
#include "bn_persistent.h"

namespace bn {
namespace {

constexpr int kR = 6;          // weight radius handled by this kernel
constexpr int kChunk = 128;    // bytes of a count vector per stage
constexpr int kChunkWords = kChunk / 4;

// ---- compile-time stencil: offsets with 0 < dx^2 + dy^2 <= R^2, grouped by d^2 -------------
template <int R>
struct Stencil {
    int n = 0, ncls = 0;
    int dx[(2 * R + 1) * (2 * R + 1)] = {};
    int dy[(2 * R + 1) * (2 * R + 1)] = {};
    int cls[(2 * R + 1) * (2 * R + 1)] = {};
    int cls_of_d2[R * R + 1] = {};
    constexpr Stencil()
    {
        for (int d = 0; d <= R * R; ++d) cls_of_d2[d] = -1;
        for (int d2 = 1; d2 <= R * R; ++d2) {
            bool any = false;
            for (int y = -R; y <= R; ++y)
                for (int x = -R; x <= R; ++x)
                    if (x * x + y * y == d2) {
                        dx[n] = x;
                        dy[n] = y;
                        cls[n] = ncls;
                        ++n;
                        any = true;
                    }
            if (any) {
                cls_of_d2[d2] = ncls;
                ++ncls;
            }
        }
    }
};
constexpr Stencil<kR> kSt{};
constexpr int kNOff = kSt.n;
constexpr int kNCls = kSt.ncls;
static_assert(kNOff == 112 && kNCls == 18, "radius-6 stencil");

// compile-time access to one offset (usable in device code)
template <int I>
struct StOff {
    static constexpr int dx = kSt.dx[I];
    static constexpr int dy = kSt.dy[I];
    static constexpr int cls = kSt.cls[I];
};

// ---- memory helpers ---------------------------------------------------------------------
__device__ __forceinline__ uint32_t ld_cg_u32(const void *p)
{
    uint32_t v;
    asm volatile("ld.global.cg.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ int ld_cg_i32(const void *p) { return (int)ld_cg_u32(p); }
__device__ __forceinline__ unsigned long long ld_cg_u64(const void *p)
{
    unsigned long long v;
    asm volatile("ld.global.cg.u64 %0, [%1];" : "=l"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ uint4 ld_cg_v4(const void *p)
{
    uint4 v;
    asm volatile("ld.global.cg.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}
__device__ __forceinline__ void st_cg_v4(void *p, uint4 v)
{
    asm volatile("st.global.cg.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w)
                 : "memory");
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ int warp_sum(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// ---- grid barrier (bounded spin) ----------------------------------------------------------
__device__ __forceinline__ bool grid_sync(GridBarrier *gb, unsigned int nblocks, int *s_err)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int *gen = &gb->gen;
        volatile unsigned int *err = &gb->error;
        const unsigned int g = *gen;
        __threadfence();
        if (atomicAdd(&gb->count, 1u) == nblocks - 1u) {
            atomicExch(&gb->count, 0u);
            __threadfence();
            atomicAdd(&gb->gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*gen == g) {
                if (*err) break;
                if (clock64() - t0 > kBarrierSpinCycles) {
                    atomicExch(&gb->error, 1u);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        *s_err = (int)*err;
    }
    __syncthreads();
    return *s_err == 0;
}

// ---- problem lookup ------------------------------------------------------------------------
__device__ __forceinline__ int find_problem(const int *start, int n, int u)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(start + mid) <= u)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int wrapi(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

// ---- stencil dot products of one proposed pixel over one chunk -----------------------------
template <int CB, int WINW, int... I>
__device__ __forceinline__ void stencil_dot(const uint32_t *centre, uint32_t d, int (&acc)[kNCls],
                                            std::integer_sequence<int, I...>)
{
    ((acc[StOff<I>::cls] = dot_word<CB>(
          d, centre[(StOff<I>::dy * WINW + StOff<I>::dx) * kChunkWords], acc[StOff<I>::cls])),
     ...);
}

struct Slot {
    int centre;   // window index of the pixel
    int j;        // couple
    int side;     // 0 = a, 1 = b
    int partner;  // partner pixel
    int cstar;    // class of the partner if it lies in the neighbourhood, else -1
};

template <int BX, int BY, int NT, int SPW, int CB>
struct Cfg {
    static constexpr int WINW = BX + 2 * kR, WINH = BY + 2 * kR;
    static constexpr int WIN = WINW * WINH;
    static constexpr int NWARPS = NT / 32;
    static constexpr int CAP = NWARPS * SPW;  // slots per round
    static constexpr int MAXSLOT = BX * BY;   // every pixel of the block
    // one stage: window chunk + partner chunks of one round of slots
    static constexpr int STAGE = (WIN + CAP) * kChunk;
    static constexpr size_t SMEM = 2 * (size_t)STAGE + MAXSLOT * sizeof(Slot) + 256;
};

// finish a couple once all its contributions have arrived: fp32 dL, flags, log, owner claim
__device__ void finalize_couple(const Problem &pb, int j, uint32_t sw, int tsplit,
                                unsigned int *bstat)
{
    int A[kNCls];
#pragma unroll
    for (int c = 0; c < kNCls; ++c) A[c] = 0;
    const int parts = 2 * tsplit;
    for (int k = 0; k < parts; ++k) {
        const int *src = pb.side_cls + ((size_t)j * parts + k) * kMaxClasses;
#pragma unroll
        for (int c = 0; c < kNCls; ++c) A[c] += ld_cg_i32(src + c);
    }
    F2 acc = {0.f, 0.f};
    float sabs = 0.f;
#pragma unroll
    for (int c = 0; c < kNCls; ++c) {
        add_weighted_i32(acc, pb.w[c], A[c]);
        sabs += pb.w[c] * fabsf((float)A[c]);
    }
    renorm(acc);
    const float dL = -pb.scale * acc.hi;
    const float S = pb.scale * sabs;
    const bool improving = (float)pb.objective * dL < 0.f;
    const bool tie = fabsf(dL) < 1e-6f * S;
    const uint32_t xs = pass_xor(pb, sw);
    const int a = (int)((uint32_t)__ldg(pb.perm + 2 * j) ^ xs);
    const int b = (int)((uint32_t)__ldg(pb.perm + 2 * j + 1) ^ xs);
    pb.log_dE[j] = dL;
    pb.log_flags[j] = kFlagValid | (improving ? kFlagImproving : 0) | (tie ? kFlagTie : 0);
    pb.log_couples[2 * j] = a;
    pb.log_couples[2 * j + 1] = b;
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

template <int BX, int BY, int NT, int SPW, int CB>
__device__ void evaluate_unit(const Problem &pb, int local_unit, uint32_t sw, int tsplit,
                              char *smem, unsigned int *bstat)
{
    using C = Cfg<BX, BY, NT, SPW, CB>;
    const int nbx = (pb.W + BX - 1) / BX;
    const int tpart = local_unit % tsplit;
    const int blk = local_unit / tsplit;
    const int x0 = (blk % nbx) * BX, y0 = (blk / nbx) * BY;
    const int nchunks = pb.row_bytes / kChunk;
    const int c0 = (int)((long long)nchunks * tpart / tsplit);
    const int c1 = (int)((long long)nchunks * (tpart + 1) / tsplit);

    Slot *slots = reinterpret_cast<Slot *>(smem + 2 * C::STAGE);
    int *s_nslot = reinterpret_cast<int *>(smem + 2 * C::STAGE + C::MAXSLOT * sizeof(Slot));
    int *s_col = s_nslot + 1;            // tile x of each window column  [WINW]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // 1. proposed pixels of the block
    if (threadIdx.x == 0) *s_nslot = 0;
    __syncthreads();
    const uint32_t xs = pass_xor(pb, sw);
    const int twoM = 2 * pb.M;
    for (int lp = threadIdx.x; lp < BX * BY; lp += NT) {
        const int x = x0 + lp % BX, y = y0 + lp / BX;
        if (x >= pb.W || y >= pb.H) continue;
        const int p = y * pb.W + x;
        const int i = __ldg(pb.perm_inv + ((uint32_t)p ^ xs));
        if (i >= twoM) continue;
        const int partner = (int)((uint32_t)__ldg(pb.perm + (i ^ 1)) ^ xs);
        if (partner >= pb.P) continue;
        Slot s;
        s.centre = (lp / BX + kR) * C::WINW + (lp % BX + kR);
        s.j = i >> 1;
        s.side = i & 1;
        s.partner = partner;
        const int ox = wrapi(partner % pb.W - x, pb.W), oy = wrapi(partner / pb.W - y, pb.H);
        const int dx = min(ox, pb.W - ox), dy = min(oy, pb.H - oy);
        const int d2 = dx * dx + dy * dy;
        s.cstar = -1;
        for (int c = 0; c < kNCls; ++c)
            if (pb.d2[c] == d2) s.cstar = c;
        slots[atomicAdd(s_nslot, 1)] = s;
    }
    for (int wx = threadIdx.x; wx < C::WINW; wx += NT) s_col[wx] = wrapi(x0 - kR + wx, pb.W);
    __syncthreads();
    const int nslot = *s_nslot;
    if (nslot == 0) return;

    uint32_t *stage[2] = {reinterpret_cast<uint32_t *>(smem),
                          reinterpret_cast<uint32_t *>(smem + C::STAGE)};
    const int parts = 2 * tsplit;

    for (int base = 0; base < nslot; base += C::CAP) {
        const int nround = min(C::CAP, nslot - base);
        int acc[SPW][kNCls];
        int corr[SPW];
#pragma unroll
        for (int k = 0; k < SPW; ++k) {
            corr[k] = 0;
#pragma unroll
            for (int c = 0; c < kNCls; ++c) acc[k][c] = 0;
        }
        auto issue = [&](int chunk, uint32_t *dst) {
            const size_t coff = (size_t)chunk * kChunk;
            for (int e = threadIdx.x; e < C::WIN * (kChunk / 16); e += NT) {
                const int wp = e / (kChunk / 16), part = e % (kChunk / 16);
                const int wx = wp % C::WINW, wy = wp / C::WINW;
                const int ty = wrapi(y0 - kR + wy, pb.H);
                const int q = ty * pb.W + s_col[wx];
                cp_async16(reinterpret_cast<char *>(dst) + (size_t)wp * kChunk + part * 16,
                           pb.counts + (size_t)q * pb.row_bytes + coff + part * 16);
            }
            for (int e = threadIdx.x; e < nround * (kChunk / 16); e += NT) {
                const int sl = e / (kChunk / 16), part = e % (kChunk / 16);
                const int q = slots[base + sl].partner;
                cp_async16(reinterpret_cast<char *>(dst) + (size_t)(C::WIN + sl) * kChunk + part * 16,
                           pb.counts + (size_t)q * pb.row_bytes + coff + part * 16);
            }
            cp_async_commit();
        };
        issue(c0, stage[0]);
        for (int c = c0; c < c1; ++c) {
            const int cur = (c - c0) & 1;
            if (c + 1 < c1) {
                issue(c + 1, stage[cur ^ 1]);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();
            const uint32_t *win = stage[cur];
#pragma unroll
            for (int k = 0; k < SPW; ++k) {
                const int sl = warp + k * C::NWARPS;
                if (sl < nround) {
                    const Slot s = slots[base + sl];
                    const uint32_t *centre = win + (size_t)s.centre * kChunkWords + lane;
                    const uint32_t kp = *centre;
                    const uint32_t kq = win[(size_t)(C::WIN + sl) * kChunkWords + lane];
                    const uint32_t d = sub_word<CB>(kq, kp);
                    corr[k] = dot_word<CB>(d, kq, corr[k]);
                    stencil_dot<CB, C::WINW>(centre, d, acc[k],
                                             std::make_integer_sequence<int, kNOff>{});
                }
            }
            __syncthreads();
        }
        // 3. per slot: reduce, remove the partner's own term, publish, finalize if last
#pragma unroll
        for (int k = 0; k < SPW; ++k) {
            const int sl = warp + k * C::NWARPS;
            if (sl >= nround) continue;
            const Slot s = slots[base + sl];
            const int cr = warp_sum(corr[k]);
            int *dst = pb.side_cls + ((size_t)s.j * parts + s.side * tsplit + tpart) * kMaxClasses;
#pragma unroll
            for (int c = 0; c < kNCls; ++c) {
                int v = warp_sum(acc[k][c]);
                if (c == s.cstar) v -= cr;
                if (lane == 0) dst[c] = v;
            }
            if (lane == 0) {
                __threadfence();
                const int arrived = atomicAdd(pb.arrivals + s.j, 1);
                if (arrived == parts - 1) {
                    __threadfence();
                    pb.arrivals[s.j] = 0;
                    finalize_couple(pb, s.j, sw, tsplit, bstat);
                }
            }
        }
        __syncthreads();
    }
}

// phase 2 for one couple (one warp); returns true (on lane 0) when the swap was applied
__device__ bool resolve_commit(const Problem &pb, int j, uint32_t sw)
{
    const int lane = threadIdx.x & 31;
    const uint32_t xs = pass_xor(pb, sw);
    const int a = (int)((uint32_t)__ldg(pb.perm + 2 * j) ^ xs);
    const int b = (int)((uint32_t)__ldg(pb.perm + 2 * j + 1) ^ xs);
    // owner claims of the previous pass (same parity as the next one) are cleared here
    if (sw > 0 && pb.mode == 0 && lane == 0) {
        const uint32_t xp = pass_xor(pb, sw - 1u);
        const int ap = (int)((uint32_t)__ldg(pb.perm + 2 * j) ^ xp);
        const int bp = (int)((uint32_t)__ldg(pb.perm + 2 * j + 1) ^ xp);
        unsigned long long *prev = pb.owner + (size_t)((sw - 1u) & 1u) * pb.P;
        if (ap < pb.P) prev[ap] = 0ull;
        if (bp < pb.P) prev[bp] = 0ull;
    }
    if (a >= pb.P || b >= pb.P) {
        if (lane == 0) {
            pb.log_dE[j] = 0.f;
            pb.log_flags[j] = 0;
            pb.log_couples[2 * j] = a;
            pb.log_couples[2 * j + 1] = b;
        }
        return false;
    }
    const uint8_t flags = (uint8_t)(ld_cg_u32(reinterpret_cast<const uint32_t *>(
                                        pb.log_flags + (j & ~3))) >>
                                    (8 * (j & 3)));
    if (!(flags & kFlagImproving)) return false;
    bool win = true;
    if (pb.mode == 0) {
        const unsigned long long key = couple_key(pb, sw, j);
        const unsigned long long *own = pb.owner + (size_t)(sw & 1u) * pb.P;
        bool lose = false;
        for (int i = lane; i < 2 * pb.n_off; i += 32) {
            const int side = i >= pb.n_off;
            const int p = side ? b : a;
            const int q = neighbour(pb, p % pb.W, p / pb.W, side ? i - pb.n_off : i);
            if (ld_cg_u64(own + q) > key) lose = true;
        }
        win = !__any_sync(0xFFFFFFFFu, lose);
    }
    if (!win) return false;
    uint8_t *ra = pb.counts + (size_t)a * pb.row_bytes;
    uint8_t *rb = pb.counts + (size_t)b * pb.row_bytes;
    for (int v = lane; v < (pb.row_bytes >> 4); v += 32) {
        const uint4 x = ld_cg_v4(ra + 16 * v), y = ld_cg_v4(rb + 16 * v);
        st_cg_v4(ra + 16 * v, y);
        st_cg_v4(rb + 16 * v, x);
    }
    if (lane == 0) {
        const int t = ld_cg_i32(pb.sidx + a);
        pb.sidx[a] = ld_cg_i32(pb.sidx + b);
        pb.sidx[b] = t;
        pb.log_flags[j] = flags | kFlagCommitted;
    }
    return lane == 0;
}

template <int BX, int BY, int NT, int SPW, int CB, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_persistent(PersistentArgs args)
{
    extern __shared__ __align__(128) char smem[];
    __shared__ int s_err;
    __shared__ unsigned int bstat[4];
    const int nblocks = gridDim.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gwarp = blockIdx.x * (NT / 32) + warp, nwarps = nblocks * (NT / 32);

    for (int it = 0; it < args.n_iter; ++it) {
        // ---- phase 1: evaluate -------------------------------------------------------------
        for (int u = blockIdx.x; u < args.total_units; u += nblocks) {
            const int pi = find_problem(args.unit_start, args.n_prob, u);
            const Problem &pb = args.probs[pi];
            const long long s = pb.ctr[0] + it;
            if (s >= pb.ctr[1]) continue;
            if (threadIdx.x < 4) bstat[threadIdx.x] = 0u;
            __syncthreads();
            evaluate_unit<BX, BY, NT, SPW, CB>(pb, u - __ldg(args.unit_start + pi), (uint32_t)s,
                                               args.tsplit, smem, bstat);
            __syncthreads();
            if (threadIdx.x < 4 && bstat[threadIdx.x])
                atomicAdd(&pb.stats[threadIdx.x], (unsigned long long)bstat[threadIdx.x]);
        }
        if (!grid_sync(args.bar, nblocks, &s_err)) return;
        // ---- phase 2: resolve + commit -------------------------------------------------------
        int cur_pi = -1;
        unsigned int mine = 0u;
        for (int g = gwarp; g < args.total_couples; g += nwarps) {
            const int pi = find_problem(args.couple_start, args.n_prob, g);
            const Problem &pb = args.probs[pi];
            const long long s = pb.ctr[0] + it;
            if (s >= pb.ctr[1]) continue;
            if (pi != cur_pi) {
                if (cur_pi >= 0 && mine && lane == 0)
                    atomicAdd(&args.probs[cur_pi].stats[kStatCommitted], (unsigned long long)mine);
                mine = 0u;
                cur_pi = pi;
            }
            if (resolve_commit(pb, g - __ldg(args.couple_start + pi), (uint32_t)s)) mine += 1u;
        }
        if (cur_pi >= 0 && mine && lane == 0)
            atomicAdd(&args.probs[cur_pi].stats[kStatCommitted], (unsigned long long)mine);
        if (!grid_sync(args.bar, nblocks, &s_err)) return;
    }
    // ---- epilogue: clear the last pass's owner claims, advance the pass counters ------------
    for (int g = gwarp; g < args.total_couples; g += nwarps) {
        const int pi = find_problem(args.couple_start, args.n_prob, g);
        const Problem &pb = args.probs[pi];
        const long long s0 = pb.ctr[0];
        const long long last = min(s0 + args.n_iter, pb.ctr[1]) - 1;
        if (last < s0 || pb.mode != 0 || lane != 0) continue;
        const int j = g - __ldg(args.couple_start + pi);
        const uint32_t xp = pass_xor(pb, (uint32_t)last);
        const int ap = (int)((uint32_t)__ldg(pb.perm + 2 * j) ^ xp);
        const int bp = (int)((uint32_t)__ldg(pb.perm + 2 * j + 1) ^ xp);
        unsigned long long *own = pb.owner + (size_t)((uint32_t)last & 1u) * pb.P;
        if (ap < pb.P) own[ap] = 0ull;
        if (bp < pb.P) own[bp] = 0ull;
    }
    if (!grid_sync(args.bar, nblocks, &s_err)) return;
    if (blockIdx.x == 0) {
        for (int pi = threadIdx.x; pi < args.n_prob; pi += NT) {
            const Problem &pb = args.probs[pi];
            const long long s0 = pb.ctr[0];
            const long long done = max(0ll, min(s0 + args.n_iter, pb.ctr[1]) - s0);
            pb.ctr[0] = s0 + done;
            pb.stats[kStatSweeps] += (unsigned long long)done;
        }
    }
}

template <int BX, int BY, int NT, int SPW, int CB, int MINB>
cudaError_t launch_cfg(const PersistentArgs &a0, int sms, cudaStream_t st, int *grid_out)
{
    using C = Cfg<BX, BY, NT, SPW, CB>;
    auto kern = k_persistent<BX, BY, NT, SPW, CB, MINB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C::SMEM);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, C::SMEM);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int grid = per_sm * sms;
    const int need = a0.total_units > a0.total_couples / (NT / 32)
                         ? a0.total_units
                         : (a0.total_couples + NT / 32 - 1) / (NT / 32);
    if (grid > need) grid = need > 0 ? need : 1;
    PersistentArgs a = a0;
    void *params[] = {&a};
    *grid_out = grid;
    return cudaLaunchCooperativeKernel((const void *)kern, dim3(grid), dim3(NT), params, C::SMEM,
                                       st);
}

}  // namespace

int persistent_units_per_problem(const Problem &h, int bx, int by, int tsplit)
{
    return ((h.W + bx - 1) / bx) * ((h.H + by - 1) / by) * tsplit;
}

bool persistent_supported(const Problem &h)
{
    return h.radius == kR && h.W >= 2 * kR + 1 && h.H >= 2 * kR + 1 && h.n_cls == kNCls &&
           h.n_off == kNOff;
}

cudaError_t launch_persistent(const PersistentArgs &a, const PersistentShape &shape, int cb,
                              int sms, cudaStream_t st)
{
    int grid = 0;
    cudaError_t e = cudaErrorInvalidValue;
#define BN_SHAPE(BX, BY, NT, SPW, MINB)                                                      \
    if (shape.bx == BX && shape.by == BY && shape.threads == NT && shape.spw == SPW)         \
        e = cb == 1 ? launch_cfg<BX, BY, NT, SPW, 1, MINB>(a, sms, st, &grid)                \
                    : launch_cfg<BX, BY, NT, SPW, 2, MINB>(a, sms, st, &grid);
    BN_PERSISTENT_SHAPES(BN_SHAPE)
#undef BN_SHAPE
    note_launches(1);
    return e;
}

}  // namespace bn
