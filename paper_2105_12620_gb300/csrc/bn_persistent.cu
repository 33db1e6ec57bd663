// bn_persistent.cu — the parallel swap optimiser (Sec. 3.4) as one cooperative, persistent
// launch that runs many passes over a batch of problems (tiles x pairs of dimensions).
//
// Per pass, three phases separated by grid barriers:
//   phase 1 (evaluate): CTAs take work units from an atomic counter.  A unit is a block of
//     BX x BY pixels of one problem and a range of 128-byte chunks of the count vectors.  The
//     CTA finds the block's proposed pixels (pixels of a valid couple of this pass).  One
//     producer warp then streams, chunk by chunk, the block's window (the block plus a halo of
//     the weight radius, wrapped on the torus) into a two-stage shared-memory ring with bulk
//     asynchronous copies (cp.async.bulk, completion on an mbarrier); the counts are stored
//     chunk-major, so every window row is one or two contiguous runs.  The producer runs one
//     unit ahead: it publishes the next unit's proposed pixels while the compute warps still
//     work on the current one.  The compute warps read their proposed pixels' partner chunks
//     straight from L2 (prefetched one chunk ahead) and accumulate, per proposed pixel p and
//     class c,
//         A_c(p) += delta_p . k_q  over q in S_c(p),   delta_p = k_partner - k_p,
//     with the 112 stencil offsets as compile-time shared-memory displacements (one IDP4A per
//     four 8-bit counts).  The partner's own term is removed and the 18 class sums are reduced
//     across the warp by a transposing butterfly and stored.
//   phase 2 (finalize): one thread per couple adds the 2 x tsplit partial class sums, computes
//     dL in fp32 (compensated), flags and logs it and, if the swap improves the objective,
//     claims the couple's pixels in the owner grid; it also clears the couple's claims of the
//     previous pass.
//   phase 3 (resolve + commit): improving couples only, one warp each: a couple is kept unless
//     an interacting improving couple (a pixel within the radius) has a higher priority; kept
//     swaps move the count vectors and the shift index.
// Data written inside the launch is read back through L2 (.cg loads) because L1 is not coherent
// across SMs.  Every wait (grid barrier, mbarrier) has a clock budget; when it runs out the
// kernel records an error, lets its own copies land (again bounded) and returns.
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
    constexpr Stencil()
    {
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
            if (any) ++ncls;
        }
    }
};
constexpr Stencil<kR> kSt{};
constexpr int kNOff = kSt.n;
constexpr int kNCls = kSt.ncls;
static_assert(kNOff == 112 && kNCls == 18, "radius-6 stencil");

template <int I>
struct StOff {
    static constexpr int dx = kSt.dx[I];
    static constexpr int dy = kSt.dy[I];
    static constexpr int cls = kSt.cls[I];
};

// ---- PTX helpers -------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait: false when the clock budget runs out
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity,
                                          long long budget = kBarrierSpinCycles)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > budget) return false;
    return true;
}
// warp-uniform bounded wait that first honours an abort raised elsewhere in the CTA
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, volatile int *s_abort)
{
    const int lane = threadIdx.x & 31;
    bool ok = __shfl_sync(0xFFFFFFFFu, lane == 0 ? *s_abort : 0, 0) == 0;
    if (ok) ok = __all_sync(0xFFFFFFFFu, mbar_wait(bar, parity));
    if (!ok && lane == 0) *s_abort = 1;
    return ok;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// ---- grid barrier (bounded spin) ----------------------------------------------------------
__device__ __forceinline__ bool grid_sync(GridBarrier *gb, unsigned int nblocks, int *s_err,
                                          long long budget = kBarrierSpinCycles)
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
                if (clock64() - t0 > budget) {
                    atomicExch(&gb->error, 1u);
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        *s_err = (int)*err;
    }
    __syncthreads();
    return *s_err == 0;
}

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

// Butterfly that sums 32 per-lane vectors and transposes them: lane l returns the warp sum of
// v[l].  16 + 8 + 4 + 2 + 1 = 31 shuffles.
__device__ __forceinline__ int transpose_reduce32(int (&v)[32], int lane)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        const bool upper = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < off; ++i) {
            const int send = upper ? v[i] : v[i + off];
            const int keep = upper ? v[i + off] : v[i];
            v[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, off);
        }
    }
    return v[0];
}


struct Slot {
    int centre;   // window index of the pixel
    int j;        // couple
    int side;     // 0 = a, 1 = b
    int partner;  // partner pixel
    int cstar;    // class of the partner if it lies in the neighbourhood, else -1
    int p;        // the pixel
};

// one work unit as published by the producer to the compute warps
struct UnitHdr {
    int nslot;    // -1: no more units in this pass
    int pi;       // problem
    int tpart;
    int c0, c1;   // chunk range
    uint32_t sw;  // pass index of the problem
    int pad[2];
};

template <int BX, int BY, int NCW, int SPW>
struct Cfg {
    static constexpr int WINW = BX + 2 * kR, WINH = BY + 2 * kR;
    static constexpr int WIN = WINW * WINH;
    static constexpr int NT = (NCW + 1) * 32;      // compute warps + one producer warp
    static constexpr int CAP = NCW * SPW;          // proposed pixels per round
    static constexpr int MAXSLOT = BX * BY;
    static constexpr int STAGE = WIN * kChunk;
    static constexpr int OFF_SLOTS = 2 * STAGE;
    static constexpr int OFF_HDR = OFF_SLOTS + 2 * MAXSLOT * (int)sizeof(Slot);
    static constexpr int OFF_BAR = (OFF_HDR + 2 * (int)sizeof(UnitHdr) + 63) / 64 * 64;
    static constexpr size_t SMEM = (size_t)OFF_BAR + 128;  // 8 mbarriers
};

// finish a couple after phase 1: fp32 dL, flags, log, owner claim (one thread); returns flags.
// Also clears the couple's claims of the previous pass (the other parity of the owner grid,
// read by the previous pass's phase 3 and next written by the next pass's phase 2).
__device__ uint8_t finalize_couple(const Problem &pb, int j, uint32_t sw, int tsplit)
{
    const int pj0 = __ldg(pb.perm + 2 * j), pj1 = __ldg(pb.perm + 2 * j + 1);
    if (sw > 0 && pb.mode == 0) {
        const uint32_t xp = pass_xor(pb, sw - 1u);
        const int ap = (int)((uint32_t)pj0 ^ xp), bp = (int)((uint32_t)pj1 ^ xp);
        unsigned long long *prev = pb.owner + (size_t)((sw - 1u) & 1u) * pb.P;
        if (ap < pb.P) prev[ap] = 0ull;
        if (bp < pb.P) prev[bp] = 0ull;
    }
    const uint32_t xs = pass_xor(pb, sw);
    const int a = (int)((uint32_t)pj0 ^ xs);
    const int b = (int)((uint32_t)pj1 ^ xs);
    pb.log_couples[2 * j] = a;
    pb.log_couples[2 * j + 1] = b;
    if (a >= pb.P || b >= pb.P) {
        pb.log_dE[j] = 0.f;
        pb.log_flags[j] = 0;
        return 0;
    }
    int A[20];
#pragma unroll
    for (int c = 0; c < 20; ++c) A[c] = 0;
    const int parts = 2 * tsplit;
    for (int k = 0; k < parts; ++k) {
        const int4 *src =
            reinterpret_cast<const int4 *>(pb.side_cls + ((size_t)j * parts + k) * kMaxClasses);
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            const int4 v = __ldcg(src + q);
            A[4 * q] += v.x;
            A[4 * q + 1] += v.y;
            A[4 * q + 2] += v.z;
            A[4 * q + 3] += v.w;
        }
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
    const uint8_t flags = kFlagValid | (improving ? kFlagImproving : 0) | (tie ? kFlagTie : 0);
    pb.log_dE[j] = dL;
    pb.log_flags[j] = flags;
    if (improving && pb.mode == 0) {
        const unsigned long long key = couple_key(pb, sw, j);
        unsigned long long *own = pb.owner + (size_t)(sw & 1u) * pb.P;
        own[a] = key;
        own[b] = key;
    }
    return flags;
}

// Per-CTA pipeline state.  Stage and slot-buffer use counters advance identically in every warp.
struct Pipe {
    uint64_t *full;    // [2] copies of a stage have landed
    uint64_t *empty;   // [2] every compute warp is done with a stage
    uint64_t *sfull;   // [2] a unit's slot list and header are ready
    uint64_t *sempty;  // [2] every compute warp is done with a slot list
    unsigned g;        // chunks streamed so far (stage = g & 1)
    unsigned ub;       // unit slot buffers used so far (buffer = ub & 1)
    unsigned issued;   // stage uses armed by the producer (for the abort path)
};

// Producer warp: takes units from the counter, publishes each unit's proposed pixels, then
// streams the unit's window chunks into the ring.
template <int BX, int BY, int NCW, int SPW>
__device__ void produce_pass(const PersistentArgs &args, int it, char *smem, Pipe &pp,
                             volatile int *s_abort)
{
    using C = Cfg<BX, BY, NCW, SPW>;
    const int lane = threadIdx.x & 31;
    for (;;) {
        int u = 0;
        if (lane == 0) u = atomicAdd(args.work + (it & 1), 1);
        u = __shfl_sync(0xFFFFFFFFu, u, 0);
        const unsigned b = pp.ub & 1u, buse = pp.ub >> 1;
        int pi = -1;
        long long s = 0;
        if (u < args.total_units) {
            pi = find_problem(args.unit_start, args.n_prob, u);
            s = args.probs[pi].ctr[0] + it;
            if (s >= args.probs[pi].ctr[1]) continue;  // problem already at its pass end
        }
        // the slot buffer must have been released by the compute warps
        if (buse >= 1 && !warp_wait(&pp.sempty[b], (buse - 1) & 1u, s_abort)) return;
        UnitHdr *hdr = reinterpret_cast<UnitHdr *>(smem + C::OFF_HDR) + b;
        Slot *slots = reinterpret_cast<Slot *>(smem + C::OFF_SLOTS) + b * C::MAXSLOT;
        if (pi < 0) {
            if (lane == 0) {
                hdr->nslot = -1;
                mbar_arrive(&pp.sfull[b]);
            }
            ++pp.ub;
            return;
        }
        const Problem &pb = args.probs[pi];
        const int tsplit = args.tsplit;
        const int lu = u - __ldg(args.unit_start + pi);
        const int nbx = (pb.W + BX - 1) / BX;
        const int tpart = lu % tsplit, blk = lu / tsplit;
        const int x0 = (blk % nbx) * BX, y0 = (blk / nbx) * BY;
        const int nchunks = pb.row_bytes / kChunk;
        const int c0 = (int)((long long)nchunks * tpart / tsplit);
        const int c1 = (int)((long long)nchunks * (tpart + 1) / tsplit);
        const uint32_t sw = (uint32_t)s;
        const uint32_t xs = pass_xor(pb, sw);
        const int twoM = 2 * pb.M;
        // proposed pixels, compacted in row-major order
        int nslot = 0;
        for (int base = 0; base < BX * BY; base += 32) {
            const int lp = base + lane;
            const int x = x0 + lp % BX, y = y0 + lp / BX;
            bool hit = false;
            Slot sl;
            if (lp < BX * BY && x < pb.W && y < pb.H) {
                const int p = y * pb.W + x;
                const int i = __ldg(pb.perm_inv + ((uint32_t)p ^ xs));
                if (i < twoM) {
                    const int partner = (int)((uint32_t)__ldg(pb.perm + (i ^ 1)) ^ xs);
                    if (partner < pb.P) {
                        hit = true;
                        sl.centre = (lp / BX + kR) * C::WINW + (lp % BX + kR);
                        sl.j = i >> 1;
                        sl.side = i & 1;
                        sl.partner = partner;
                        sl.p = p;
                        const int ox = wrapi(partner % pb.W - x, pb.W);
                        const int oy = wrapi(partner / pb.W - y, pb.H);
                        const int dx = min(ox, pb.W - ox), dy = min(oy, pb.H - oy);
                        const int d2 = dx * dx + dy * dy;
                        sl.cstar = -1;
                        for (int c = 0; c < kNCls; ++c)
                            if (pb.d2[c] == d2) sl.cstar = c;
                    }
                }
            }
            const unsigned m = __ballot_sync(0xFFFFFFFFu, hit);
            if (hit) slots[nslot + __popc(m & ((1u << lane) - 1u))] = sl;
            nslot += __popc(m);
        }
        if (lane == 0) {
            hdr->nslot = nslot;
            hdr->pi = pi;
            hdr->tpart = tpart;
            hdr->c0 = c0;
            hdr->c1 = c1;
            hdr->sw = sw;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&pp.sfull[b]);
        ++pp.ub;
        // stream the unit, one round of proposed pixels at a time
        const int xa = x0 - kR, xb = x0 + BX + kR;  // window columns [xa, xb), W >= xb - xa
        for (int base = 0; base < nslot; base += C::CAP) {
            const int nround = min(C::CAP, nslot - base);
            const uint32_t tx = (uint32_t)C::WIN * kChunk;
            for (int c = c0; c < c1; ++c) {
                const unsigned g = pp.g, st = g & 1u, use = g >> 1;
                if (use >= 1 && !warp_wait(&pp.empty[st], (use - 1) & 1u, s_abort)) return;
                if (__shfl_sync(0xFFFFFFFFu, lane == 0 ? *s_abort : 0, 0)) return;
                char *dst = smem + st * C::STAGE;
                if (lane == 0) mbar_arrive_expect_tx(&pp.full[st], tx);
                __syncwarp();
                for (int wy = lane; wy < C::WINH; wy += 32) {
                    const int ty = wrapi(y0 - kR + wy, pb.H);
                    const uint8_t *rowp = chunk_ptr(pb, ty * pb.W, c);
                    char *d = dst + (size_t)wy * C::WINW * kChunk;
                    if (xa < 0) {
                        bulk_g2s(d, rowp + (size_t)(pb.W + xa) * kChunk, (uint32_t)(-xa) * kChunk,
                                 &pp.full[st]);
                        bulk_g2s(d + (size_t)(-xa) * kChunk, rowp, (uint32_t)xb * kChunk,
                                 &pp.full[st]);
                    } else if (xb > pb.W) {
                        bulk_g2s(d, rowp + (size_t)xa * kChunk, (uint32_t)(pb.W - xa) * kChunk,
                                 &pp.full[st]);
                        bulk_g2s(d + (size_t)(pb.W - xa) * kChunk, rowp,
                                 (uint32_t)(xb - pb.W) * kChunk, &pp.full[st]);
                    } else {
                        bulk_g2s(d, rowp + (size_t)xa * kChunk, (uint32_t)(xb - xa) * kChunk,
                                 &pp.full[st]);
                    }
                }
                pp.issued = g + 1;
                ++pp.g;
            }
        }
    }
}

// Compute warps: for every unit of the pass and every round of its proposed pixels, warp w
// accumulates the proposed pixels w, w + NCW, ... over the unit's chunks, then stores the class
// sums of each (the partner's own term removed).
template <int BX, int BY, int NCW, int SPW, int CB>
__device__ void consume_pass(const PersistentArgs &args, char *smem, Pipe &pp,
                             volatile int *s_abort)
{
    using C = Cfg<BX, BY, NCW, SPW>;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        const unsigned b = pp.ub & 1u, buse = pp.ub >> 1;
        if (!warp_wait(&pp.sfull[b], buse & 1u, s_abort)) return;
        const UnitHdr hdr = reinterpret_cast<const UnitHdr *>(smem + C::OFF_HDR)[b];
        const Slot *slots = reinterpret_cast<const Slot *>(smem + C::OFF_SLOTS) + b * C::MAXSLOT;
        if (hdr.nslot < 0) {
            __syncwarp();
            if (lane == 0) mbar_arrive(&pp.sempty[b]);
            ++pp.ub;
            return;
        }
        const Problem &pb = args.probs[hdr.pi];
        const int parts = 2 * args.tsplit;
        for (int base = 0; base < hdr.nslot; base += C::CAP) {
            const int nround = min(C::CAP, hdr.nslot - base);
            int acc[SPW][kNCls];
            uint32_t kq_next[SPW];
            const uint32_t *prow[SPW];  // the partner's words of this lane, chunk 0
#pragma unroll
            for (int k = 0; k < SPW; ++k) {
#pragma unroll
                for (int c = 0; c < kNCls; ++c) acc[k][c] = 0;
                const int sl = warp + k * NCW;
                prow[k] = nullptr;
                kq_next[k] = 0u;
                if (sl < nround) {
                    prow[k] = reinterpret_cast<const uint32_t *>(
                                  chunk_ptr(pb, slots[base + sl].partner, 0)) + lane;
                    kq_next[k] = __ldcg(prow[k] + (size_t)hdr.c0 * pb.P * kChunkWords);
                }
            }
            for (int c = hdr.c0; c < hdr.c1; ++c) {
                const unsigned g = pp.g, st = g & 1u, use = g >> 1;
                if (!warp_wait(&pp.full[st], use & 1u, s_abort)) return;
                const uint32_t *win = reinterpret_cast<const uint32_t *>(smem + st * C::STAGE);
#pragma unroll
                for (int k = 0; k < SPW; ++k) {
                    const int sl = warp + k * NCW;
                    if (sl < nround) {
                        const uint32_t kq = kq_next[k];
                        if (c + 1 < hdr.c1)
                            kq_next[k] = __ldcg(prow[k] + (size_t)(c + 1) * pb.P * kChunkWords);
                        const uint32_t *centre =
                            win + (size_t)slots[base + sl].centre * kChunkWords + lane;
                        const uint32_t d = sub_word<CB>(kq, *centre);
                        stencil_dot<CB, C::WINW>(centre, d, acc[k],
                                                 std::make_integer_sequence<int, kNOff>{});
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&pp.empty[st]);
                ++pp.g;
            }
#pragma unroll
            for (int k = 0; k < SPW; ++k) {
                const int sl = warp + k * NCW;
                if (sl >= nround) continue;
                const Slot s = slots[base + sl];
                // rare: the partner lies in the neighbourhood; remove its own term, recomputed
                // from the counts over the unit's chunks
                int corr = 0;
                if (s.cstar >= 0) {
                    for (int c = hdr.c0; c < hdr.c1; ++c) {
                        const uint32_t kq = __ldcg(reinterpret_cast<const unsigned int *>(
                                                       chunk_ptr(pb, s.partner, c)) + lane);
                        const uint32_t kp = __ldcg(reinterpret_cast<const unsigned int *>(
                                                       chunk_ptr(pb, s.p, c)) + lane);
                        corr = dot_word<CB>(sub_word<CB>(kq, kp), kq, corr);
                    }
                }
                int v[32];
#pragma unroll
                for (int c = 0; c < 32; ++c)
                    v[c] = c < kNCls ? acc[k][c] - (c == s.cstar ? corr : 0) : 0;
                const int sum = transpose_reduce32(v, lane);
                if (lane < kNCls)
                    pb.side_cls[((size_t)s.j * parts + s.side * args.tsplit + hdr.tpart) *
                                    kMaxClasses + lane] = sum;
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&pp.sempty[b]);
        ++pp.ub;
    }
}

__device__ bool resolve_commit(const Problem &pb, int j, uint32_t sw, uint8_t flags)
{
    const int lane = threadIdx.x & 31;
    const uint32_t xs = pass_xor(pb, sw);
    const int a = (int)((uint32_t)__ldg(pb.perm + 2 * j) ^ xs);
    const int b = (int)((uint32_t)__ldg(pb.perm + 2 * j + 1) ^ xs);
    if (pb.mode == 0) {
        const unsigned long long key = couple_key(pb, sw, j);
        const unsigned long long *own = pb.owner + (size_t)(sw & 1u) * pb.P;
        const int ax = a % pb.W, ay = a / pb.W, bx = b % pb.W, by = b / pb.W;
        constexpr int kPer = (2 * kNOff + 31) / 32;
        unsigned long long v[kPer];
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int i = lane + 32 * k;
            v[k] = 0ull;
            if (i < 2 * kNOff) {
                const int side = i >= kNOff;
                const int q = side ? neighbour(pb, bx, by, i - kNOff) : neighbour(pb, ax, ay, i);
                v[k] = __ldcg(own + q);
            }
        }
        bool lose = false;
#pragma unroll
        for (int k = 0; k < kPer; ++k) lose |= v[k] > key;
        if (__any_sync(0xFFFFFFFFu, lose)) return false;
    }
    for (int vi = lane; vi < (pb.row_bytes >> 4); vi += 32) {
        uint4 *pa = vec_ptr(pb, a, vi), *pbp = vec_ptr(pb, b, vi);
        const uint4 x = __ldcg(pa), y = __ldcg(pbp);
        __stcg(pa, y);
        __stcg(pbp, x);
    }
    if (lane == 0) {
        const int t = __ldcg(pb.sidx + a);
        pb.sidx[a] = __ldcg(pb.sidx + b);
        pb.sidx[b] = t;
        pb.log_flags[j] = flags | kFlagCommitted;
    }
    return true;
}

template <int BX, int BY, int NCW, int SPW, int CB, int MINB>
__global__ void __launch_bounds__((NCW + 1) * 32, MINB) k_persistent(PersistentArgs args)
{
    using C = Cfg<BX, BY, NCW, SPW>;
    extern __shared__ __align__(128) char smem_raw[];
    __shared__ int s_err;
    __shared__ int s_abort;
    char *smem = smem_raw;
    const int nblocks = gridDim.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gwarp = blockIdx.x * (C::NT / 32) + warp, nwarps = nblocks * (C::NT / 32);

    Pipe pp;
    pp.full = reinterpret_cast<uint64_t *>(smem + C::OFF_BAR);
    pp.empty = pp.full + 2;
    pp.sfull = pp.full + 4;
    pp.sempty = pp.full + 6;
    pp.g = 0;
    pp.ub = 0;
    pp.issued = 0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&pp.full[i], 1);
            mbar_init(&pp.empty[i], NCW);
            mbar_init(&pp.sfull[i], 1);
            mbar_init(&pp.sempty[i], NCW);
        }
        mbar_init_fence();
        s_abort = 0;
        s_err = 0;
    }
    __syncthreads();

    for (int it = 0; it < args.n_iter; ++it) {
        // ---- phase 1: evaluate (units from an atomic counter) -------------------------------
        if (warp == NCW)
            produce_pass<BX, BY, NCW, SPW>(args, it, smem, pp, &s_abort);
        else
            consume_pass<BX, BY, NCW, SPW, CB>(args, smem, pp, &s_abort);
        __syncthreads();
        if (s_abort) {
            if (threadIdx.x == 0) atomicExch(&args.bar->error, 2u);
            break;
        }
        if (!grid_sync(args.bar, nblocks, &s_err)) break;
        // ---- phase 2: finalize (one thread per couple) ---------------------------------------
        if (blockIdx.x == 0 && threadIdx.x == 0) args.work[(it + 1) & 1] = 0;
        for (int base = gwarp * 32; base < args.total_couples; base += nwarps * 32) {
            const int g = base + lane;
            int pi = -1;
            uint8_t f = 0;
            if (g < args.total_couples) {
                pi = find_problem(args.couple_start, args.n_prob, g);
                const Problem &pb = args.probs[pi];
                const long long s = pb.ctr[0] + it;
                if (s < pb.ctr[1])
                    f = finalize_couple(pb, g - __ldg(args.couple_start + pi), (uint32_t)s,
                                        args.tsplit);
                else
                    pi = -1;
            }
            // warp-aggregated counters, one group of lanes per problem
            const unsigned grp = __match_any_sync(0xFFFFFFFFu, pi);
            const unsigned nv = __popc(__ballot_sync(0xFFFFFFFFu, f & kFlagValid) & grp);
            const unsigned ni = __popc(__ballot_sync(0xFFFFFFFFu, f & kFlagImproving) & grp);
            const unsigned nt = __popc(__ballot_sync(0xFFFFFFFFu, f & kFlagTie) & grp);
            if (pi >= 0 && lane == __ffs(grp) - 1) {
                unsigned long long *st = args.probs[pi].stats;
                if (nv) atomicAdd(&st[kStatValid], (unsigned long long)nv);
                if (ni) atomicAdd(&st[kStatImproving], (unsigned long long)ni);
                if (nt) atomicAdd(&st[kStatTies], (unsigned long long)nt);
            }
        }
        if (!grid_sync(args.bar, nblocks, &s_err)) break;
        // ---- phase 3: resolve + commit -------------------------------------------------------
        // 32 couples per warp step: one flag load each, then the improving ones one by one
        for (int base = gwarp * 32; base < args.total_couples; base += nwarps * 32) {
            const int g = base + lane;
            int pi = 0, j = 0;
            uint8_t f = 0;
            uint32_t sw = 0;
            if (g < args.total_couples) {
                pi = find_problem(args.couple_start, args.n_prob, g);
                const Problem &pb = args.probs[pi];
                const long long s = pb.ctr[0] + it;
                if (s < pb.ctr[1]) {
                    j = g - __ldg(args.couple_start + pi);
                    sw = (uint32_t)s;
                    f = (uint8_t)(__ldcg(reinterpret_cast<const unsigned int *>(pb.log_flags +
                                                                               (j & ~3))) >>
                                  (8 * (j & 3)));
                }
            }
            unsigned m = __ballot_sync(0xFFFFFFFFu, (f & kFlagImproving) != 0);
            while (m) {
                const int l = __ffs(m) - 1;
                m &= m - 1u;
                const int lpi = __shfl_sync(0xFFFFFFFFu, pi, l);
                const int lj = __shfl_sync(0xFFFFFFFFu, j, l);
                const uint32_t lsw = __shfl_sync(0xFFFFFFFFu, sw, l);
                const uint8_t lf = (uint8_t)__shfl_sync(0xFFFFFFFFu, (int)f, l);
                if (resolve_commit(args.probs[lpi], lj, lsw, lf) && lane == 0)
                    atomicAdd(&args.probs[lpi].stats[kStatCommitted], 1ull);
            }
        }
        if (!grid_sync(args.bar, nblocks, &s_err)) break;
    }
    if (s_abort || s_err) {
        // let this CTA's own copies land before it leaves (bounded)
        if (warp == NCW && lane == 0) {
            const unsigned issued = pp.issued;
            for (unsigned g = (issued >= 2u ? issued - 2u : 0); g < issued; ++g)
                mbar_wait(&pp.full[g % 2u], (g / 2u) & 1u);
        }
        __syncthreads();
        return;
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
        for (int pi = threadIdx.x; pi < args.n_prob; pi += C::NT) {
            const Problem &pb = args.probs[pi];
            const long long s0 = pb.ctr[0];
            const long long done = max(0ll, min(s0 + args.n_iter, pb.ctr[1]) - s0);
            pb.ctr[0] = s0 + done;
            pb.stats[kStatSweeps] += (unsigned long long)done;
        }
    }
}

// after a persistent launch: a barrier timeout or an aborted pipeline becomes a sticky error of
// every problem of the launch (read back as BN_ERR_TIMEOUT)
__global__ void k_fold_error(const GridBarrier *gb, const Problem *probs, int n_prob)
{
    const unsigned int err = gb->error;
    if (!err) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_prob; i += gridDim.x * blockDim.x)
        atomicOr(&probs[i].stats[kStatError], (unsigned long long)err);
}

// Runs the kernel's own bounded waits on conditions that cannot occur, with a short budget:
// which = 0: a grid barrier that waits for one more block than the grid has;
// which = 1: an mbarrier that nobody arrives at.  result[0] = 1 when the wait ran out.
__global__ void k_selftest_wait(int which, long long budget, GridBarrier *gb, int *result)
{
    __shared__ int s_err;
    __shared__ uint64_t bar;
    bool ok;
    if (which == 0) {
        if (threadIdx.x == 0) s_err = 0;
        __syncthreads();
        ok = grid_sync(gb, gridDim.x + 1u, &s_err, budget);
    } else {
        if (threadIdx.x == 0) {
            mbar_init(&bar, 1);
            mbar_init_fence();
        }
        __syncthreads();
        ok = mbar_wait(&bar, 0u, budget);
        __syncthreads();
    }
    if (threadIdx.x == 0 && blockIdx.x == 0) result[0] = ok ? 0 : 1;
}

template <int BX, int BY, int NCW, int SPW, int CB, int MINB>
cudaError_t launch_cfg(const PersistentArgs &a0, int sms, cudaStream_t st)
{
    using C = Cfg<BX, BY, NCW, SPW>;
    constexpr size_t smem_bytes = C::SMEM;
    auto kern = k_persistent<BX, BY, NCW, SPW, CB, MINB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_bytes);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, C::NT, smem_bytes);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int grid = per_sm * sms;
    const int need = a0.total_units > a0.total_couples / (C::NT / 32)
                         ? a0.total_units
                         : (a0.total_couples + C::NT / 32 - 1) / (C::NT / 32);
    if (grid > need) grid = need > 0 ? need : 1;
    PersistentArgs a = a0;
    void *params[] = {&a};
    return cudaLaunchCooperativeKernel((const void *)kern, dim3(grid), dim3(C::NT), params,
                                       smem_bytes, st);
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

bool persistent_shape_fits(const Problem &h, const PersistentShape &s)
{
    // a window row must wrap at most once
    return persistent_supported(h) && h.W >= s.bx + 2 * kR;
}

cudaError_t launch_fold_error(const GridBarrier *gb, const Problem *probs, int n_prob,
                              cudaStream_t st)
{
    k_fold_error<<<1, 128, 0, st>>>(gb, probs, n_prob);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_selftest_wait(int which, long long budget, GridBarrier *gb, int *result,
                                 cudaStream_t st)
{
    k_selftest_wait<<<which == 0 ? 2 : 1, 64, 0, st>>>(which, budget, gb, result);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_persistent(const PersistentArgs &a, const PersistentShape &shape, int cb,
                              int sms, cudaStream_t st)
{
    cudaError_t e = cudaErrorInvalidValue;
#define BN_SHAPE(BX, BY, NCW, KMAX, MINB)                                                     \
    if (shape.bx == BX && shape.by == BY && shape.threads == (NCW + 1) * 32 &&                \
        shape.spw == KMAX)                                                                     \
        e = cb == 1 ? launch_cfg<BX, BY, NCW, KMAX, 1, MINB>(a, sms, st)                     \
                    : launch_cfg<BX, BY, NCW, KMAX, 2, MINB>(a, sms, st);
    BN_PERSISTENT_SHAPES(BN_SHAPE)
#undef BN_SHAPE
    note_launches(1);
    return e;
}

}  // namespace bn
