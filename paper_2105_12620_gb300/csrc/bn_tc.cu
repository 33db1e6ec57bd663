// bn_tc.cu — one pass of the parallel swap optimiser (Sec. 3.4) with the stencil of Eq. 1 on the
// fifth-generation tensor cores (tcgen05.mma, accumulators in tensor memory).
//
// For every proposed pixel n of a pass (one side of a valid couple) let delta_n =
// k_partner(n) - k_n.  The class sums of a couple j = (a, b) are A_c = S_c(a) + S_c(b) with
//   S_c(n) = sum over pixels q at squared torus distance c from n, q != partner(n), of
//            delta_n . k_q,
// i.e. selected entries of the product D = K . Delta^T of count vectors (rows q) and deltas
// (rows n).  The tile is cut into patches of 16 x 8 pixels.  Per patch the tensor core forms
// D[q][n] for the patch's 128 pixels q (M = 128) and the proposed pixels n within the weight
// radius of it (the patch's list, at most 192 per product), accumulating over all T integrands
// in tensor memory; about a fifth of the entries lie inside the radius and are kept.  The f16
// operands are exact (counts <= 64, |delta| <= 64) and the f32 sums stay within 2^24
// (T N^2 <= 2^24 for 8-bit counts), so every kept entry is an exact integer.
//
// A pass:
//   k_tc_lists     couples of the pass as in the plain schedule; each proposed pixel is appended
//                  to the list of every patch within the radius of it; its class sums cleared
//   k_tc_stencil   one CTA per SM over the patches, warp-specialised:
//                    8 producer warps   count bytes -> shared memory (cp.async), converted in
//                                       place to f16 in the 128-byte swizzled K-major layout,
//                                       deltas formed on the way; stages of 64 integrands
//                    1 MMA warp         four tcgen05.mma (K = 16 each) per stage
//                    4 epilogue warps   tensor memory -> registers; entries inside the radius
//                                       go to per-pixel class sums in shared memory, then to
//                                       the global class sums (integer atomics)
//                  four stages in a ring, two accumulator buffers in tensor memory
//   k_tc_finalize  change of Eq. 1 from the class sums, flags and pixel claims
//   then the resolve and commit kernels of the plain schedule.
// Every wait is bounded; a wait that runs out raises the problems' error word and the CTA
// drains its copies and products, frees its tensor memory and returns.
#include "bn_launch.h"
#include "bn_tcgen05.cuh"

namespace bn {
namespace {

constexpr int kPW = 16, kPH = 8, kTcM = kPW * kPH;  // patch: M = 128 pixels
constexpr int kNB = 192;                             // listed pixels per product (N)
constexpr int kStages = 4;                           // ring of 64-integrand stages
constexpr int kLook = 2;                             // stages in flight per producer thread
constexpr int kAStage = kTcM * 128;                  // 16 KB: 128 rows x 64 f16
constexpr int kBStage = kNB * 128;                   // 24 KB: 192 rows x 64 f16
constexpr int kStageBytes = kAStage + kBStage;
constexpr int kEpiWarps = 4, kProdWarps = 8;
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kProdThreads = kProdWarps * 32;
constexpr int kMmaWarp = kEpiWarps + kProdWarps;
constexpr int kTcThreads = (kMmaWarp + 1) * 32;      // 416
constexpr uint32_t kTmemCols = 512, kTmemBuf = 256;  // two accumulator buffers
constexpr int kTabMax = 65;                          // squared distances 0..64 (radius <= 8)
constexpr long long kSpin = 1ll << 31;               // ~1 s at 2 GHz
constexpr unsigned long long kErrTc = 3ull;

// shared memory layout (offsets from a 1024-byte aligned base)
constexpr int kOffAcc = kStages * kStageBytes;        // int32 [kNB][32] class sums
constexpr int kOffCol = kOffAcc + kNB * 32 * 4;       // int4  [kNB] (x, y, partner, slot)
constexpr int kOffTab = kOffCol + kNB * 16;           // int32 [80] class of a squared distance
constexpr int kOffBar = kOffTab + 80 * 4;             // mbarriers
constexpr int kNBars = 2 * kStages + 5;
constexpr int kOffMisc = kOffBar + kNBars * 8;        // tensor-memory base, abort flag
constexpr int kSmemBytes = kOffMisc + 16 + 1024;
static_assert(kStageBytes % 1024 == 0 && kAStage % 1024 == 0, "stage alignment");
static_assert(kOffBar % 8 == 0, "mbarrier alignment");
static_assert(kSmemBytes <= 227 * 1024, "shared memory");

struct TcArgs {
    const Problem *probs;
    int n_prob;
    const int *unit_start;  // [n_prob + 1] prefix sums of patches
    int total_units;
};

// ---- PTX helpers ----------------------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc::saddr(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::saddr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(tc::saddr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait; false when the budget runs out (the abort flag is then raised) or another role
// has aborted
__device__ __forceinline__ bool tc_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (clock64() - t0 > kSpin) {
            *abort_flag = 1;
            return false;
        }
    }
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst),
                 "l"(__cvta_generic_to_global(src))
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
// named barrier of the epilogue warps
__device__ __forceinline__ void epi_sync()
{
    asm volatile("bar.sync 1, %0;" ::"n"(kEpiThreads) : "memory");
}
// the same, returning whether any epilogue thread passed true
__device__ __forceinline__ bool epi_any(bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(kEpiThreads)
        : "memory");
    return r != 0;
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

// four bytes -> two f16x2 (bytes 0,1 and 2,3); the bytes are read as 1024 + byte and bias
// (1024, or 1152 for deltas stored offset by 128) is subtracted, so the values are exact
__device__ __forceinline__ void bytes_to_h2(uint32_t x, uint32_t bias2, uint32_t &lo, uint32_t &hi)
{
    const uint32_t a = __byte_perm(x, 0x64646464u, 0x4140);
    const uint32_t b = __byte_perm(x, 0x64646464u, 0x4342);
    asm("sub.f16x2 %0, %1, %2;" : "=r"(lo) : "r"(a), "r"(bias2));
    asm("sub.f16x2 %0, %1, %2;" : "=r"(hi) : "r"(b), "r"(bias2));
}
constexpr uint32_t kBiasCount = 0x64006400u;  // f16x2 (1024, 1024)
constexpr uint32_t kBiasDelta = 0x64806480u;  // f16x2 (1152, 1152)

// The unit decode shared by the three roles: the same global sequence of patches and of
// products (jobs) on every role, from values that do not change during the launch.
struct Unit {
    const Problem *pb;
    int pid, cnt, x0, y0;
    uint32_t xs;
};
__device__ __forceinline__ Unit decode_unit(const TcArgs &args, int u, int &pi)
{
    pi = find_problem(args.unit_start, args.n_prob, u);
    Unit d;
    d.pb = args.probs + pi;
    const Problem &pb = *d.pb;
    d.pid = u - __ldg(args.unit_start + pi);
    const long long s = pb.ctr[0];
    int c = 0;
    if (s < pb.ctr[1]) {
        c = pb.tc_cnt[d.pid];
        c = c < pb.tc_cap ? c : pb.tc_cap;
    }
    d.cnt = c;
    d.x0 = (d.pid % pb.tc_npx) * kPW;
    d.y0 = (d.pid / pb.tc_npx) * kPH;
    d.xs = pass_xor(pb, (uint32_t)s);
    return d;
}

// proposed pixel and partner of a listed slot 2 j + side
__device__ __forceinline__ void slot_pixels(const Problem &pb, uint32_t xs, int slot, int &p,
                                            int &partner)
{
    const int j = slot >> 1;
    const int a = (int)((uint32_t)pb.perm[2 * j] ^ xs);
    const int b = (int)((uint32_t)pb.perm[2 * j + 1] ^ xs);
    p = (slot & 1) ? b : a;
    partner = (slot & 1) ? a : b;
}

// row kinds of a producer task
enum : int { kRowNone = 0, kRowCount = 1, kRowDelta = 2, kRowZero = 3 };

// In place: the raw bytes of one row (64 counts, or 64 partner then 64 own counts) become its
// 64 f16 in swizzled order.  r7: the row's swizzle phase (row index mod 8).
__device__ __forceinline__ void convert_row(int kind, char *row, uint32_t r7)
{
    if (kind == kRowNone) return;
    uint4 out[8];
    uint4 *raw = reinterpret_cast<uint4 *>(row);
    if (kind == kRowCount) {
        uint4 v[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = raw[i];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const uint32_t w0 = (j & 1) ? v[j >> 1].z : v[j >> 1].x;
            const uint32_t w1 = (j & 1) ? v[j >> 1].w : v[j >> 1].y;
            bytes_to_h2(w0, kBiasCount, out[j].x, out[j].y);
            bytes_to_h2(w1, kBiasCount, out[j].z, out[j].w);
        }
    } else if (kind == kRowDelta) {
        uint4 v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = raw[i];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const uint4 pa = v[j >> 1], se = v[4 + (j >> 1)];
            const uint32_t p0 = (j & 1) ? pa.z : pa.x, p1 = (j & 1) ? pa.w : pa.y;
            const uint32_t s0 = (j & 1) ? se.z : se.x, s1 = (j & 1) ? se.w : se.y;
            // signed byte differences (|d| <= 64), offset by 128 to read them unsigned
            const uint32_t d0 = __vsub4(p0, s0) ^ 0x80808080u;
            const uint32_t d1 = __vsub4(p1, s1) ^ 0x80808080u;
            bytes_to_h2(d0, kBiasDelta, out[j].x, out[j].y);
            bytes_to_h2(d1, kBiasDelta, out[j].z, out[j].w);
        }
    } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) out[j] = make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) raw[j ^ r7] = out[j];
}

// ---- producer warps -----------------------------------------------------------------------
__device__ void tc_produce(const TcArgs &args, char *smem, uint64_t *full, uint64_t *empty,
                           volatile int *abort_flag)
{
    const int pt = threadIdx.x - kEpiThreads;  // 0 .. kProdThreads - 1
    const uint32_t sbase = tc::saddr(smem);
    uint32_t g = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < args.total_units && ok; u += gridDim.x) {
        int pi;
        const Unit d = decode_unit(args, u, pi);
        if (d.cnt <= 0) continue;
        const Problem &pb = *d.pb;
        const int nks = pb.row_bytes >> 6;
        const size_t plane = (size_t)pb.P << 7;
        const int32_t *list = pb.tc_list + (size_t)d.pid * pb.tc_cap;
        for (int n0 = 0; n0 < d.cnt && ok; n0 += kNB) {
            const int nn = d.cnt - n0 < kNB ? d.cnt - n0 : kNB;
            const int npad = (nn + 15) & ~15;
            // this thread's rows: A rows 0..127 then B rows 0..npad-1
            int kind[2];
            const uint8_t *src0[2], *src1[2];
            uint32_t roff[2];
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int row = pt + t * kProdThreads;
                kind[t] = kRowNone;
                src0[t] = src1[t] = nullptr;
                roff[t] = 0;
                if (row < kTcM) {
                    roff[t] = (uint32_t)((row >> 3) * 1024 + (row & 7) * 128);
                    const int qx = d.x0 + (row & 15), qy = d.y0 + (row >> 4);
                    if (qx < pb.W && qy < pb.H) {
                        kind[t] = kRowCount;
                        src0[t] = pb.counts + ((size_t)(qy * pb.W + qx) << 7);
                    } else {
                        kind[t] = kRowZero;
                    }
                } else if (row < kTcM + npad) {
                    const int n = row - kTcM;
                    roff[t] = (uint32_t)(kAStage + (n >> 3) * 1024 + (n & 7) * 128);
                    if (n < nn) {
                        int p, partner;
                        slot_pixels(pb, d.xs, list[n0 + n], p, partner);
                        kind[t] = kRowDelta;
                        src0[t] = pb.counts + ((size_t)partner << 7);
                        src1[t] = pb.counts + ((size_t)p << 7);
                    } else {
                        kind[t] = kRowZero;
                    }
                }
            }
            for (int ks = 0; ks < nks + kLook; ++ks) {
                if (ks < nks) {
                    const uint32_t gi = g + (uint32_t)ks;
                    const uint32_t slot = gi % kStages, use = gi / kStages;
                    if (!tc_wait(&empty[slot], (use & 1u) ^ 1u, abort_flag)) {
                        ok = false;
                        break;
                    }
                    const uint32_t st = sbase + slot * kStageBytes;
                    const size_t off = (size_t)(ks >> 1) * plane + (size_t)(ks & 1) * 64;
#pragma unroll
                    for (int t = 0; t < 2; ++t) {
                        if (kind[t] == kRowCount || kind[t] == kRowDelta) {
#pragma unroll
                            for (int i = 0; i < 4; ++i)
                                cp_async16(st + roff[t] + 16 * i, src0[t] + off + 16 * i);
                        }
                        if (kind[t] == kRowDelta) {
#pragma unroll
                            for (int i = 0; i < 4; ++i)
                                cp_async16(st + roff[t] + 64 + 16 * i, src1[t] + off + 16 * i);
                        }
                    }
                }
                cp_async_commit();
                if (ks >= kLook) {
                    cp_async_wait<kLook>();
                    const uint32_t gi = g + (uint32_t)(ks - kLook);
                    const uint32_t slot = gi % kStages;
                    char *st = smem + slot * kStageBytes;
#pragma unroll
                    for (int t = 0; t < 2; ++t)
                        convert_row(kind[t], st + roff[t], (roff[t] >> 7) & 7u);
                    tc::fence_async_smem();
                    mbar_arrive(&full[slot]);
                }
            }
            g += (uint32_t)nks;
        }
    }
    cp_async_wait<0>();
}

// ---- MMA warp -------------------------------------------------------------------------------
__device__ void tc_mma(const TcArgs &args, char *smem, uint64_t *full, uint64_t *empty,
                       uint64_t *tfull, uint64_t *tempty, uint64_t *done, uint32_t tmem,
                       volatile int *abort_flag, volatile int *no_abort)
{
    const int lane = threadIdx.x & 31;
    const uint32_t sbase = tc::saddr(smem);
    uint32_t g = 0, jb = 0;
    bool ok = true, issued = false;
    for (int u = blockIdx.x; u < args.total_units && ok; u += gridDim.x) {
        int pi;
        const Unit d = decode_unit(args, u, pi);
        if (d.cnt <= 0) continue;
        const int nks = d.pb->row_bytes >> 6;
        for (int n0 = 0; n0 < d.cnt && ok; n0 += kNB) {
            const int nn = d.cnt - n0 < kNB ? d.cnt - n0 : kNB;
            const int npad = (nn + 15) & ~15;
            const uint32_t buf = jb & 1u;
            ok = __all_sync(0xFFFFFFFFu, tc_wait(&tempty[buf], ((jb >> 1) & 1u) ^ 1u, abort_flag));
            if (!ok) break;
            tc::fence_after_sync();
            const uint32_t dt = tmem + buf * kTmemBuf;
            const uint32_t idesc = tc::idesc_f16_f32(kTcM, npad);
            for (int ks = 0; ks < nks; ++ks) {
                const uint32_t slot = g % kStages, use = g / kStages;
                ok = __all_sync(0xFFFFFFFFu, tc_wait(&full[slot], use & 1u, abort_flag));
                if (!ok) break;
                tc::fence_after_sync();
                if (lane == 0) {
                    const uint32_t a0 = sbase + slot * kStageBytes, b0 = a0 + kAStage;
#pragma unroll
                    for (int k16 = 0; k16 < 4; ++k16)
                        tc::mma_f16(dt, tc::sw128_desc(a0, k16), tc::sw128_desc(b0, k16), idesc,
                                    (ks | k16) != 0);
                    tc::mma_commit(&empty[slot]);
                }
                __syncwarp();
                issued = true;
                ++g;
            }
            if (!ok) break;
            if (lane == 0) tc::mma_commit(&tfull[buf]);
            __syncwarp();
            ++jb;
        }
    }
    // every product issued has completed before tensor memory is released
    if (issued) {
        if (lane == 0) tc::mma_commit(done);
        __syncwarp();
        tc_wait(done, 0u, no_abort);
    }
}

// ---- epilogue warps -------------------------------------------------------------------------
__device__ void tc_epilogue(const TcArgs &args, char *smem, uint64_t *tfull, uint64_t *tempty,
                            uint32_t tmem, volatile int *abort_flag)
{
    const int et = threadIdx.x;  // 0 .. 127: tensor-memory lane = patch pixel
    const int w = et >> 5;
    int32_t *acc = reinterpret_cast<int32_t *>(smem + kOffAcc);
    int4 *col = reinterpret_cast<int4 *>(smem + kOffCol);
    int32_t *tab = reinterpret_cast<int32_t *>(smem + kOffTab);
    uint32_t jb = 0;
    int cur = -1;
    bool ok = true;
    for (int u = blockIdx.x; u < args.total_units && ok; u += gridDim.x) {
        int pi;
        const Unit d = decode_unit(args, u, pi);
        const Problem &pb = *d.pb;
        if (d.cnt > 0 && pi != cur) {  // class of each squared distance of this problem
            epi_sync();
            for (int i = et; i < kTabMax; i += kEpiThreads) tab[i] = -1;
            epi_sync();
            if (et < pb.n_cls) tab[pb.d2[et]] = et;
            epi_sync();
            cur = pi;
        }
        const int qx = d.x0 + (et & 15), qy = d.y0 + (et >> 4);
        const bool qin = qx < pb.W && qy < pb.H;
        const int qpix = qy * pb.W + qx;
        const int W = pb.W, H = pb.H, hw = pb.W >> 1, hh = pb.H >> 1;
        const int r2 = pb.radius * pb.radius, ncls = pb.n_cls;
        const int32_t *list = pb.tc_list + (size_t)d.pid * pb.tc_cap;
        for (int n0 = 0; n0 < d.cnt; n0 += kNB) {
            const int nn = d.cnt - n0 < kNB ? d.cnt - n0 : kNB;
            const int npad = (nn + 15) & ~15;
            const uint32_t buf = jb & 1u;
            for (int n = et; n < nn; n += kEpiThreads) {
                const int slot = list[n0 + n];
                int p, partner;
                slot_pixels(pb, d.xs, slot, p, partner);
                col[n] = make_int4(p % W, p / W, partner, slot);
            }
            for (int e = et; e < nn * 8; e += kEpiThreads)
                reinterpret_cast<int4 *>(acc)[e] = make_int4(0, 0, 0, 0);
            epi_sync();
            const bool wok = tc_wait(&tfull[buf], (jb >> 1) & 1u, abort_flag);
            if (epi_any(!wok)) {
                ok = false;
                break;
            }
            tc::fence_after_sync();
            for (int c0 = 0; c0 < npad; c0 += 32) {
                uint32_t v[32];
                tc::tmem_ld32(tmem + buf * kTmemBuf + (uint32_t)c0 + ((uint32_t)(w * 32) << 16),
                              v);
                if (qin) {
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const int n = c0 + i;
                        if (n < nn) {
                            const int4 ci = col[n];
                            int dx = qx - ci.x, dy = qy - ci.y;
                            dx += dx < -hw ? W : 0;
                            dx -= dx > hw ? W : 0;
                            dy += dy < -hh ? H : 0;
                            dy -= dy > hh ? H : 0;
                            const int d2 = dx * dx + dy * dy;  // |dx| <= W/2, |dy| <= H/2
                            if (d2 <= r2) {
                                const int c = tab[d2];  // -1 for d2 = 0 and empty classes
                                if (c >= 0 && qpix != ci.z)
                                    atomicAdd(&acc[n * 32 + c],
                                              __float2int_rn(__uint_as_float(v[i])));
                            }
                        }
                    }
                }
            }
            tc::fence_before_sync();
            mbar_arrive(&tempty[buf]);
            epi_sync();
            for (int e = et; e < nn * 32; e += kEpiThreads) {
                const int c = e & 31;
                if (c < ncls) {
                    const int val = acc[e];
                    if (val) atomicAdd(pb.side_cls + (size_t)col[e >> 5].w * kMaxClasses + c, val);
                }
            }
            epi_sync();
            ++jb;
        }
        if (!ok) break;
        if (et == 0 && d.cnt > 0) pb.tc_cnt[d.pid] = 0;  // cleared for the next pass
    }
}

__global__ void __launch_bounds__(kTcThreads, 1) k_tc_stencil(TcArgs args)
{
    extern __shared__ unsigned char smem_raw[];
    char *smem = reinterpret_cast<char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kOffBar);
    uint64_t *full = bars, *empty = bars + kStages;
    uint64_t *tfull = bars + 2 * kStages, *tempty = tfull + 2, *done = tempty + 2;
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(smem + kOffMisc);
    volatile int *s_abort = reinterpret_cast<volatile int *>(smem + kOffMisc + 4);
    volatile int *s_zero = reinterpret_cast<volatile int *>(smem + kOffMisc + 8);  // stays 0
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages; ++i) {
            mbar_init(&full[i], kProdThreads);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&tfull[i], 1);
            mbar_init(&tempty[i], kEpiThreads);
        }
        mbar_init(done, 1);
        *s_abort = 0;
        *s_zero = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        tc::tmem_alloc(s_tmem, kTmemCols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *s_tmem;
    if (warp < kEpiWarps)
        tc_epilogue(args, smem, tfull, tempty, tmem, s_abort);
    else if (warp < kMmaWarp)
        tc_produce(args, smem, full, empty, s_abort);
    else
        tc_mma(args, smem, full, empty, tfull, tempty, done, tmem, s_abort, s_zero);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, kTmemCols);
    }
    if (threadIdx.x == 0 && *s_abort)
        for (int i = 0; i < args.n_prob; ++i) atomicExch(args.probs[i].stats + kStatError, kErrTc);
}

// ---- pass setup and finish ------------------------------------------------------------------
constexpr int kListThreads = 256;
constexpr int kMaxMet = 5;  // distinct patch columns (rows) within a radius <= 8 of a pixel

__device__ __forceinline__ void note_patch(int (&idx)[kMaxMet], int (&dist)[kMaxMet], int &n,
                                           int i, int ad)
{
    for (int k = 0; k < n; ++k)
        if (idx[k] == i) {
            dist[k] = ad < dist[k] ? ad : dist[k];
            return;
        }
    if (n < kMaxMet) {
        idx[n] = i;
        dist[n] = ad;
        ++n;
    }
}

__global__ void __launch_bounds__(kListThreads) k_tc_lists(const Problem *probs)
{
    const Problem &pb = probs[blockIdx.y];
    const long long s = pb.ctr[0];
    if (s >= pb.ctr[1]) return;
    const int j = blockIdx.x * kListThreads + threadIdx.x;
    if (j >= pb.M) return;
    const uint32_t xs = pass_xor(pb, (uint32_t)s);
    const int a = (int)((uint32_t)pb.perm[2 * j] ^ xs);
    const int b = (int)((uint32_t)pb.perm[2 * j + 1] ^ xs);
    if (a >= pb.P || b >= pb.P) return;
    int4 *cls = reinterpret_cast<int4 *>(pb.side_cls + (size_t)j * 2 * kMaxClasses);
#pragma unroll
    for (int i = 0; i < 2 * kMaxClasses / 4; ++i) cls[i] = make_int4(0, 0, 0, 0);
    const int r = pb.radius, r2 = r * r;
    for (int side = 0; side < 2; ++side) {
        const int p = side ? b : a, px = p % pb.W, py = p / pb.W;
        // distinct patch columns (rows) met by x in [px - r, px + r] (y likewise), torus-wrapped,
        // with the smallest |offset| that reaches each (a walk can leave a patch and come back
        // to it on a narrow torus, so every earlier entry is checked)
        int xi[kMaxMet], xd[kMaxMet], yi[kMaxMet], yd[kMaxMet], nx = 0, ny = 0;
        for (int dd = -r; dd <= r; ++dd) {
            const int ad = dd < 0 ? -dd : dd;
            note_patch(xi, xd, nx, wrap_add(px, dd, pb.W) / kPW, ad);
            note_patch(yi, yd, ny, wrap_add(py, dd, pb.H) / kPH, ad);
        }
        for (int u = 0; u < nx; ++u)
            for (int v = 0; v < ny; ++v) {
                if (xd[u] * xd[u] + yd[v] * yd[v] > r2) continue;  // patch out of reach
                const int pid = yi[v] * pb.tc_npx + xi[u];
                const int pos = atomicAdd(pb.tc_cnt + pid, 1);
                if (pos < pb.tc_cap) pb.tc_list[(size_t)pid * pb.tc_cap + pos] = 2 * j + side;
            }
    }
}

__global__ void __launch_bounds__(kListThreads) k_tc_finalize(const Problem *probs)
{
    const Problem &pb = probs[blockIdx.y];
    const long long s = pb.ctr[0];
    if (s >= pb.ctr[1]) return;
    __shared__ unsigned int bstat[4];
    if (threadIdx.x < 4) bstat[threadIdx.x] = 0u;
    __syncthreads();
    const int j = blockIdx.x * kListThreads + threadIdx.x;
    if (j < pb.M) {
        const uint32_t sw = (uint32_t)s;
        const uint32_t xs = pass_xor(pb, sw);
        const int a = (int)((uint32_t)pb.perm[2 * j] ^ xs);
        const int b = (int)((uint32_t)pb.perm[2 * j + 1] ^ xs);
        float dL = 0.f, S = 0.f;
        uint8_t flags = 0;
        if (a < pb.P && b < pb.P) {
            const int32_t *ca = pb.side_cls + (size_t)j * 2 * kMaxClasses;
            const int32_t *cb = ca + kMaxClasses;
            int A[kMaxClasses];
#pragma unroll
            for (int c = 0; c < kMaxClasses; ++c) A[c] = c < pb.n_cls ? ca[c] + cb[c] : 0;
            couple_delta(pb, A, dL, S);
            const bool improving = (float)pb.objective * dL < 0.f;
            const bool tie = fabsf(dL) < 1e-6f * S;
            flags = kFlagValid | (improving ? kFlagImproving : 0) | (tie ? kFlagTie : 0);
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
        pb.log_dE[j] = dL;
        pb.log_flags[j] = flags;
        pb.log_couples[2 * j] = a;
        pb.log_couples[2 * j + 1] = b;
    }
    __syncthreads();
    if (threadIdx.x < 4 && bstat[threadIdx.x])
        atomicAdd(&pb.stats[threadIdx.x], (unsigned long long)bstat[threadIdx.x]);
}

}  // namespace

bool tc_supported(const Problem &h)
{
    return h.count_bytes == 1 && h.radius >= 1 && h.radius <= 8 && h.W >= 2 * h.radius + 1 &&
           h.H >= 2 * h.radius + 1 && h.n_cls <= kMaxClasses && h.row_bytes % 128 == 0;
}

int tc_units_per_problem(const Problem &h) { return h.tc_npx * h.tc_npy; }

cudaError_t prepare_tc()
{
    return cudaFuncSetAttribute(k_tc_stencil, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kSmemBytes);
}

cudaError_t launch_tc_sweep(const TcLaunch &tl, cudaStream_t st, KernelTimer *tm)
{
    const dim3 gl((tl.max_M + kListThreads - 1) / kListThreads, tl.n_prob);
    k_tc_lists<<<gl, kListThreads, 0, st>>>(tl.dprob);
    if (tl.total_units > 0) {
        const TcArgs a{tl.dprob, tl.n_prob, tl.unit_start, tl.total_units};
        const int grid = tl.total_units < tl.sms ? tl.total_units : tl.sms;
        const bool timed = tm && tm->enabled;
        if (timed) tm->begin(kKTcStencil, st);
        k_tc_stencil<<<grid, kTcThreads, kSmemBytes, st>>>(a);
        if (timed) tm->end(st);
        note_launches(1);
    }
    k_tc_finalize<<<gl, kListThreads, 0, st>>>(tl.dprob);
    note_launches(2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_resolve_commit(SweepLaunch{tl.dprob, tl.n_prob, tl.max_M, 1}, st);
}

}  // namespace bn
