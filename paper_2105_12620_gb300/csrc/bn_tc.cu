// bn_tc.cu — one pass of the parallel swap optimiser (Sec. 3.4) with the stencil of Eq. 1 on the
// fifth-generation tensor cores (tcgen05.mma; A operand and accumulators in tensor memory).
//
// For every proposed pixel n of a pass (one side of a valid couple) let delta_n =
// k_partner(n) - k_n.  The class sums of a couple j = (a, b) are A_c = S_c(a) + S_c(b) with
//   S_c(n) = sum over pixels q at squared torus distance c from n, q != partner(n), of
//            delta_n . k_q,
// i.e. selected entries of the product D = K . Delta^T of count vectors (rows q) and deltas
// (rows n).  The tile is cut into patches of 16 x 8 pixels.  Per patch the tensor core forms
// D[q][n] for the patch's 128 pixels q (M = 128) and the proposed pixels n within the weight
// radius of it (the patch's list, at most 160 per product), accumulating over all T integrands
// in tensor memory; about a fifth of the entries lie inside the radius and are kept.
//
// Exactness.  The A operand holds the centred counts c_q = k_q - N/2 (|c| <= N/2), the B operand
// the deltas (|delta| <= N), both exact in f16.  The integrands of a product are summed in
// accumulator rounds of R stages of 64, R 64 N^2 <= 2^25: every partial sum of a round is an
// integer of magnitude at most R 64 (N/2) N <= 2^24, exact in the f32 accumulators, and the
// rounds add as integers (one round when T N^2 <= 2^25).  The centring adds
// (N/2) (sum_t delta_n[t]) x |S_c(n)| to S_c(n); side b carries -delta_a and on a torus
// |S_c(a) \ b| = |S_c(b) \ a|, so the two corrections cancel in A_c, whose magnitude is at most
// 2 x 12 x T (N/2) N = 12 T N^2 (at most 12 pixels share a squared distance within radius 8):
// below 2^31 for T N^2 <= 2^27, the plan-time limit.
//
// A pass:
//   k_tc_lists     one warp per couple: its class sums cleared, its f16 delta row k_b - k_a
//                  written per stage of 64 integrands, each of its pixels appended to the list
//                  of every patch within the radius
//   k_tc_stencil   one CTA of 24 warps per SM over the patches:
//                    A loader (1 thread)  one TMA box per 128-byte count chunk: the patch's 128
//                                         pixels x 128 bytes (zero outside the tile), 128-byte
//                                         swizzle, into a ring of four boxes
//                    8 converter warps    thread = patch pixel = tensor-memory lane (two warps
//                                         per lane quadrant, one half of the integrands each):
//                                         its chunk -> exact centred f16 -> tensor memory
//                                         (tcgen05.st), 64 integrands per slot
//                    4 producer warps     cp.async of the listed couples' delta rows (B)
//                                         straight into the 128-byte swizzled K-major layout;
//                                         a ring of six stages of 64 integrands, each an A slot
//                                         and a delta tile, full when the converters and every
//                                         producer thread's copies have arrived
//                    3 MMA warps          stage g issued by warp g mod 3: four tcgen05.mma (A
//                                         from tensor memory, B from shared memory, K = 16)
//                                         into one of two accumulators (M = 128, N <= 160),
//                                         which the epilogue zeroes as it reads them; a
//                                         product takes one accumulator per round
//                    8 epilogue warps     16 accumulator columns per warp and step, transposed
//                                         through shared memory 32 columns at a time; for
//                                         radius 6 each warp owns whole distance classes and
//                                         sums them over the stencil offsets of every listed
//                                         pixel (compile-time offsets), then adds them to the
//                                         couple's class sums in global memory; other radii
//                                         and narrow tiles go through a class table and
//                                         shared-memory atomics
//   k_tc_finalize  change of Eq. 1 from the class sums, flags and pixel claims
//   then the resolve and commit kernels of the plain schedule.
// Every wait is bounded; a wait that runs out raises the problems' error word and the CTA
// drains its copies and products, frees its tensor memory and returns.
#include <utility>

#include <cuda.h>

#include "bn_launch.h"
#include "bn_tcgen05.cuh"

namespace bn {
namespace {

constexpr int kPW = 16, kPH = 8, kTcM = kPW * kPH;  // patch: M = 128 pixels
constexpr int kNB = 160;                             // listed pixels per product (N)
constexpr int kABoxes = 3;                           // ring of count boxes (TMA)
constexpr int kStages = 6;                           // ring of stages of 64 integrands: an A slot in
                                                     // tensor memory and a delta tile in shared
                                                     // memory each, one full and one empty barrier
constexpr int kBoxBytes = kTcM * 128;                // 16 KB: 128 pixels x 128 count bytes
constexpr int kBStageBytes = kNB * 128;              // 20 KB: 160 rows x 64 f16
constexpr int kEpiWarps = 8, kConvWarps = 8, kProdWarps = 4;
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kConvWarp0 = kEpiWarps;                // converter warp c: lane quadrant c mod 4,
                                                     // integrand half c / 4 of every slot
constexpr int kProdWarp0 = kConvWarp0 + kConvWarps;
constexpr int kLoadWarp = kProdWarp0 + kProdWarps;
constexpr int kMmaWarp0 = kLoadWarp + 1;
constexpr int kMmaWarps = 3;                         // stage g is issued by MMA warp g mod 3
constexpr int kTcThreads = (kMmaWarp0 + kMmaWarps) * 32;  // 608
constexpr int kProdThreads = kProdWarps * 32;
constexpr int kBTasks = kNB * 8 / kProdThreads;      // 16-byte pieces per producer thread
constexpr uint32_t kTmemCols = 512, kAccCols = kNB;  // accumulators at columns 0 and 160
constexpr uint32_t kColA = 2 * kAccCols;             // A slot s at column 320 + 32 s
constexpr int kTabMax = 65;                          // squared distances 0..64 (radius <= 8)
constexpr long long kSpin = 1ll << 31;               // ~1 s at 2 GHz
constexpr unsigned long long kErrTc = 3ull;
constexpr int kFlushBatch = 5;                       // class-sum rows sent per batch
constexpr int kTensorMapBytes = 128;                 // one CUtensorMap per problem
constexpr int kUnitTab = 64;                         // patches of one CTA per launch (a pass with
                                                     // more is split over launches)
static_assert(kConvWarp0 % 4 == 0, "lane quadrants of the converter warps");
static_assert(kColA + 32 * kStages <= kTmemCols, "tensor memory");
constexpr int kProdRowStep = kProdThreads / 8;       // rows between a producer thread's tasks
static_assert(kBTasks * kProdThreads == 8 * kNB && kProdRowStep % 8 == 0, "producer rows");

// shared memory layout (offsets from a 1024-byte aligned base)
constexpr int kOffA = 0;                                    // count boxes, swizzled
constexpr int kOffB = kOffA + kABoxes * kBoxBytes;          // delta stages, swizzled
constexpr int kOffDt = kOffB + kStages * kBStageBytes;      // epilogue: int32 [32][128] transpose
constexpr int kDtBytes = 32 * kTcM * 4;
constexpr int kAccStride = 19;                              // class sums of one listed pixel
constexpr int kOffAcc6 = kOffDt + kDtBytes;                 // int32 [kNB][kAccStride]: class sums
constexpr int kAcc6Bytes = kNB * kAccStride * 4;            //   of a product's pixels (radius 6)
// the table paths' class sums, int32 [kNB][32], overlay the transpose and kOffAcc6 (a product
// uses one path; products are separated by epilogue barriers)
constexpr int kOffCol = kOffAcc6 + kAcc6Bytes;              // int4 [2][kNB] x 2: listed pixels
constexpr int kOffTab = kOffCol + 2 * 2 * kNB * 16;         // int32 [80] class of a squared distance
constexpr int kOffTab2 = kOffTab + 80 * 4;                  // int8 [2-D offset] class (table path)
constexpr int kTab2Max = 1664;                              // (2 (16 + 8) + 1) x (2 (8 + 8) + 1)
constexpr int kOffUnits = kOffTab2 + kTab2Max;              // TcUnit [kUnitTab]: this CTA's patches
constexpr int kOffBar = kOffUnits + kUnitTab * 64;          // mbarriers
constexpr int kNBars = 2 * kABoxes + 2 * kStages + 4 + kMmaWarps;
constexpr int kOffMisc = kOffBar + kNBars * 8;              // tensor-memory base, abort flags
constexpr int kSmemBytes = kOffMisc + 16 + 1024;
static_assert(kNB * 32 * 4 <= kDtBytes + kAcc6Bytes, "class sums of the table paths");
static_assert(kOffB % 1024 == 0 && kBStageBytes % 1024 == 0 && kOffDt % 16 == 0, "alignment");
static_assert(kOffUnits % 16 == 0 && kOffBar % 8 == 0, "table and mbarrier alignment");
static_assert(kSmemBytes <= 227 * 1024, "shared memory");

struct TcArgs {
    const Problem *probs;
    int n_prob;
    const int4 *units;      // [all patches] (problem, patch, x0, y0)
    int unit_begin;         // this launch's patches: unit_begin .. unit_begin + unit_count - 1,
    int unit_count;         //   CTA c taking the contiguous run from unit_begin + c * per
    int per;
    const char *tmaps;      // [n_prob] tensor maps of the count planes (kTensorMapBytes each)
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
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::saddr(bar)),
                 "r"(bytes)
                 : "memory");
}
// test for the completion of the phase of the given parity; the thread may be suspended in
// hardware (no instructions issued) for up to kSuspendNs while the phase is incomplete
constexpr uint32_t kSuspendNs = 100000;
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(tc::saddr(bar)), "r"(parity), "r"(kSuspendNs)
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
// the same for a whole warp: true only if every lane's wait succeeded
__device__ __forceinline__ bool tc_wait_warp(uint64_t *bar, uint32_t parity,
                                             volatile int *abort_flag)
{
    return __all_sync(0xFFFFFFFFu, tc_wait(bar, parity, abort_flag));
}
// integer add to global memory without a return value
__device__ __forceinline__ void red_add_global(int32_t *p, int v)
{
    // no compiler memory barrier: nothing in the kernel reads these sums
    asm volatile("red.global.add.s32 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "r"(v));
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint64_t policy)
{
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(dst),
                 "l"(__cvta_generic_to_global(src)), "l"(policy)
                 : "memory");
}
// one arrival on *bar once every cp.async this thread issued before has completed (the
// barrier's count includes this arrival: no pending-count increment)
__device__ __forceinline__ void cp_async_arrive(uint64_t *bar)
{
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(tc::saddr(bar))
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;" ::: "memory");
}
// L2 cache policies: data read once (the count boxes) is evicted first, so that the delta rows,
// which several patches read, stay in L2
__device__ __forceinline__ uint64_t policy_evict_first()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_last()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
// 4-D tiled TMA load into shared memory, completion counted in bytes on *bar
__device__ __forceinline__ void tma_load_4d(void *dst, const char *tmap, int c0, int c1, int c2,
                                            int c3, uint64_t *bar, uint64_t policy)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        ".L2::cache_hint [%0], [%1, {%2, %3, %4, %5}], [%6], %7;" ::"r"(tc::saddr(dst)),
        "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(tc::saddr(bar)), "l"(policy)
        : "memory");
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

// f16x2 of an unsigned 16-bit pair below 1024: each half read as 1024 + value (exact)
constexpr uint32_t kH2Magic = 0x64006400u;
__device__ __forceinline__ uint32_t h2_sub(uint32_t a, uint32_t b)
{
    uint32_t r;
    asm("sub.f16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}
// four bytes -> two f16x2 (bytes 0,1 and 2,3), each byte read as 1024 + byte; bias2 is
// subtracted, so the values (byte + 1024 - bias) are exact
__device__ __forceinline__ void bytes_to_h2(uint32_t x, uint32_t bias2, uint32_t &lo, uint32_t &hi)
{
    lo = h2_sub(__byte_perm(x, 0x64646464u, 0x4140), bias2);
    hi = h2_sub(__byte_perm(x, 0x64646464u, 0x4342), bias2);
}
// four byte differences a - b -> two f16x2: both read as 1024 + byte, then subtracted
__device__ __forceinline__ void bytes_sub_h2(uint32_t a, uint32_t b, uint32_t &lo, uint32_t &hi)
{
    lo = h2_sub(__byte_perm(a, 0x64646464u, 0x4140), __byte_perm(b, 0x64646464u, 0x4140));
    hi = h2_sub(__byte_perm(a, 0x64646464u, 0x4342), __byte_perm(b, 0x64646464u, 0x4342));
}

// stages of 64 integrands of a problem's count rows
__host__ __device__ __forceinline__ int tc_stages(const Problem &pb)
{
    return pb.row_bytes / (64 * pb.count_bytes);
}

// The CTA's patches in order, with the fields of their problems the roles need, decoded once
// per launch into shared memory by all threads at the start: every role walks the same sequence
// of patches and products without a global-memory load on the way.
struct TcUnit {
    int pi, pid, cnt, xy;    // problem, patch, listed pixels of this pass, x0 | y0 << 16
    int wh, geom, nr, M;     // W | H << 16; row_bytes | count_bytes << 16;
                             // N | radius << 16 | classes << 24; couples per pass
    const int4 *list;        // the patch's list of proposed pixels
    const uint16_t *delta;   // the problem's per-pass delta rows
    int32_t *side;           // the problem's class sums
    int flags;               // kUnitTable: 2-D table path holds; kUnitStatic6: radius-6 path;
                             // accumulator rounds per product << 8
    int kper;                // stages per accumulator round (exact f32 partial sums)
};
static_assert(sizeof(TcUnit) == 64, "unit table entry");
constexpr int kUnitTable = 1, kUnitStatic6 = 2;
struct Unit {
    const TcUnit *t;
    int pid, cnt, x0, y0;
};
__device__ __forceinline__ Unit unit_at(const TcUnit *utab, int k, int &pi)
{
    const TcUnit *t = utab + k;
    pi = t->pi;
    Unit d;
    d.t = t;
    d.pid = t->pid;
    d.cnt = t->cnt;
    d.x0 = t->xy & 0xFFFF;
    d.y0 = t->xy >> 16;
    return d;
}
__device__ __forceinline__ int unit_w(const Unit &d) { return d.t->wh & 0xFFFF; }
__device__ __forceinline__ int unit_h(const Unit &d) { return d.t->wh >> 16; }
__device__ __forceinline__ int unit_row_bytes(const Unit &d) { return d.t->geom & 0xFFFF; }
__device__ __forceinline__ int unit_count_bytes(const Unit &d) { return d.t->geom >> 16; }
// stages of 64 integrands of the patch's count rows
__device__ __forceinline__ int unit_stages(const Unit &d)
{
    return unit_row_bytes(d) / (64 * unit_count_bytes(d));
}
// stages per accumulator round: the most R with R 64 N^2 <= 2^25, at most all of them
__host__ __device__ __forceinline__ int tc_round_stages(int N, int stages)
{
    const long long r = (1ll << 25) / (64ll * N * N);
    return r < 1 ? 1 : (r < stages ? (int)r : stages);
}

// 2-D class table of the epilogue's table path: offsets (dx, dy) from a proposed pixel to a
// patch pixel, |dx| <= 16 + r, |dy| <= 8 + r, row-major with row length 2 (16 + r) + 1
__host__ __device__ __forceinline__ int tab2_dx(int r) { return 16 + r; }
__host__ __device__ __forceinline__ int tab2_dy(int r) { return 8 + r; }
__host__ __device__ __forceinline__ int tab2_w(int r) { return 2 * (16 + r) + 1; }
// the table path holds when the torus is wide enough that a proposed pixel's offset from the
// patch centre, taken as the min-image, is its true offset (below half a side): W > 2 (8 + r),
// H > 2 (4 + r)
__host__ __device__ __forceinline__ bool tab2_ok(int W, int H, int r)
{
    return W > 2 * (8 + r) && H > 2 * (4 + r);
}

// ---- compile-time stencil of radius 6: offsets with 0 < dx^2 + dy^2 <= 36, by class ----------
struct Stencil6 {
    int n = 0, ncls = 0;
    int dx[169] = {}, dy[169] = {}, cls[169] = {}, d2[32] = {}, mult[32] = {};
    constexpr Stencil6()
    {
        for (int dd = 1; dd <= 36; ++dd) {
            bool any = false;
            for (int y = -6; y <= 6; ++y)
                for (int x = -6; x <= 6; ++x)
                    if (x * x + y * y == dd) {
                        dx[n] = x;
                        dy[n] = y;
                        cls[n] = ncls;
                        ++mult[ncls];
                        ++n;
                        any = true;
                    }
            if (any) d2[ncls++] = dd;
        }
    }
};
constexpr Stencil6 kSt6{};
constexpr int kCls6 = 18;
static_assert(kSt6.n == 112 && kSt6.ncls == kCls6, "radius-6 stencil");

// The 18 classes split over the 8 epilogue warps (largest multiplicity first, each to the warp
// with the fewest offsets so far): every warp owns whole classes, at most 16 offsets.
constexpr int kGrpMaxOff = 16, kGrpMaxCls = 4;
struct Groups6 {
    int n[kEpiWarps] = {}, ncls[kEpiWarps] = {};
    int cls[kEpiWarps][kGrpMaxCls] = {};
    int dx[kEpiWarps][kGrpMaxOff] = {}, dy[kEpiWarps][kGrpMaxOff] = {},
        k[kEpiWarps][kGrpMaxOff] = {};
    constexpr Groups6()
    {
        int load[kEpiWarps] = {}, owner[kCls6] = {};
        bool used[kCls6] = {};
        for (int it = 0; it < kCls6; ++it) {
            int best = 0, bm = -1;
            for (int c = 0; c < kCls6; ++c)
                if (!used[c] && kSt6.mult[c] > bm) {
                    bm = kSt6.mult[c];
                    best = c;
                }
            used[best] = true;
            int b = 0;
            for (int i = 1; i < kEpiWarps; ++i)
                if (load[i] < load[b]) b = i;
            load[b] += bm;
            owner[best] = b;
            cls[b][ncls[b]++] = best;
        }
        for (int o = 0; o < kSt6.n; ++o) {
            const int c = kSt6.cls[o], b = owner[c];
            int kk = 0;
            for (int t = 0; t < ncls[b]; ++t)
                if (cls[b][t] == c) kk = t;
            dx[b][n[b]] = kSt6.dx[o];
            dy[b][n[b]] = kSt6.dy[o];
            k[b][n[b]] = kk;
            ++n[b];
        }
    }
    constexpr int max_n() const
    {
        int m = 0;
        for (int i = 0; i < kEpiWarps; ++i) m = n[i] > m ? n[i] : m;
        return m;
    }
    constexpr int max_cls() const
    {
        int m = 0;
        for (int i = 0; i < kEpiWarps; ++i) m = ncls[i] > m ? ncls[i] : m;
        return m;
    }
};
constexpr Groups6 kG6{};
static_assert(kG6.max_n() <= kGrpMaxOff && kG6.max_cls() <= kGrpMaxCls, "class groups");

// one offset of warp E's classes: the transposed accumulator row of patch pixel p + offset, if
// that pixel is in the patch and is not the partner, added to its class sum
template <int E, int I>
__device__ __forceinline__ void g6_add(const int32_t *dtc, int plx, int ply, int plane, int lane,
                                       int (&a)[kGrpMaxCls])
{
    if constexpr (I < kG6.n[E]) {
        constexpr int dx = kG6.dx[E][I], dy = kG6.dy[E][I], k = kG6.k[E][I];
        const int lx = plx + dx, ly = ply + dy;
        const int q = ly * kPW + lx;
        const bool in = (unsigned)lx < (unsigned)kPW && (unsigned)ly < (unsigned)kPH && q != plane;
        // unconditional load; a lane outside the patch reads its own bank (row lane)
        const int x = dtc[in ? q : lane];
        a[k] += in ? x : 0;
    }
}
// warp E's class K of the listed pixel, stored in the pixel's row of class sums (each class of
// each listed pixel has one writer: the owning warp's lane)
template <int E, int K>
__device__ __forceinline__ void g6_store(const int (&a)[kGrpMaxCls], int32_t *accrow)
{
    if constexpr (K < kG6.ncls[E]) {
        constexpr int c = kG6.cls[E][K];
        accrow[c] = a[K];
    }
}
template <int E, int... I>
__device__ __forceinline__ void g6_sum(const int32_t *dtc, int4 c1, int lane, int32_t *accrow,
                                       std::integer_sequence<int, I...>)
{
    int a[kGrpMaxCls] = {0, 0, 0, 0};
    (g6_add<E, I>(dtc, c1.x, c1.y, c1.z, lane, a), ...);
    g6_store<E, 0>(a, accrow);
    g6_store<E, 1>(a, accrow);
    g6_store<E, 2>(a, accrow);
    g6_store<E, 3>(a, accrow);
}
// warp w's classes for the listed pixel of this lane
__device__ __forceinline__ void g6_warp(int w, const int32_t *dtc, int4 c1, int lane,
                                        int32_t *accrow)
{
    using Seq = std::make_integer_sequence<int, kGrpMaxOff>;
    switch (w) {
    case 0: g6_sum<0>(dtc, c1, lane, accrow, Seq{}); break;
    case 1: g6_sum<1>(dtc, c1, lane, accrow, Seq{}); break;
    case 2: g6_sum<2>(dtc, c1, lane, accrow, Seq{}); break;
    case 3: g6_sum<3>(dtc, c1, lane, accrow, Seq{}); break;
    case 4: g6_sum<4>(dtc, c1, lane, accrow, Seq{}); break;
    case 5: g6_sum<5>(dtc, c1, lane, accrow, Seq{}); break;
    case 6: g6_sum<6>(dtc, c1, lane, accrow, Seq{}); break;
    default: g6_sum<7>(dtc, c1, lane, accrow, Seq{}); break;
    }
}
// a product's class sums sent to the couples' class sums in global memory: warp w takes the
// listed pixels w, w + 8, ..., lane = class, so each reduction covers one pixel's 18
// contiguous sums (the b side carries -delta); the loads of a batch are issued before its
// reductions
__device__ __forceinline__ void g6_flush(const int32_t *acc, const int4 *col1, int nn, int w,
                                         int lane, int32_t *side)
{
    constexpr int kB = 4;
    for (int n0 = w; n0 < nn; n0 += kEpiWarps * kB) {
        int v[kB], slot[kB];
#pragma unroll
        for (int t = 0; t < kB; ++t) {
            const int n = n0 + kEpiWarps * t;
            const bool on = n < nn && lane < kCls6;
            v[t] = on ? acc[n * kAccStride + lane] : 0;
            slot[t] = on ? col1[n].w : 0;
        }
#pragma unroll
        for (int t = 0; t < kB; ++t)
            if (v[t])
                red_add_global(side + (size_t)slot[t] * kMaxClasses + lane,
                               (slot[t] & 1) ? -v[t] : v[t]);
    }
}

// the problem's classes are those of the static stencil (squared distances in order)
template <int C>
struct D2Of6 {
    static constexpr int v = kSt6.d2[C];
};
template <int... C>
__device__ __forceinline__ bool classes_match6(const int32_t *d2, std::integer_sequence<int, C...>)
{
    return ((d2[C] == D2Of6<C>::v) && ...);
}

// ---- A loader (one thread) -------------------------------------------------------------------
// For every product, one TMA box per 128-byte count chunk: the patch's 16 x 8 pixels x 128
// bytes (8-bit counts: 128 integrands; 16-bit: 64), zero outside the tile.
__device__ void tc_load_a(const TcArgs &args, const TcUnit *utab, int nu, char *smem,
                          uint64_t *a_full, uint64_t *a_empty, volatile int *abort_flag,
                          volatile int *no_abort)
{
    uint32_t g = 0;
    bool ok = true;
    const uint64_t pol = policy_evict_first();
    for (int ku = 0; ku < nu && ok; ++ku) {
        int pi;
        const Unit d = unit_at(utab, ku, pi);
        if (d.cnt <= 0) continue;
        const int nbox = unit_row_bytes(d) >> 7;
        const char *tmap = args.tmaps + (size_t)pi * kTensorMapBytes;
        for (int n0 = 0; n0 < d.cnt && ok; n0 += kNB)
            for (int c = 0; c < nbox; ++c) {
                const uint32_t slot = g % kABoxes, use = g / kABoxes;
                if (!tc_wait(&a_empty[slot], (use & 1u) ^ 1u, abort_flag)) {
                    ok = false;
                    break;
                }
                mbar_arrive_expect_tx(&a_full[slot], kBoxBytes);
                tma_load_4d(smem + kOffA + slot * kBoxBytes, tmap, 0, d.x0, d.y0, c,
                            &a_full[slot], pol);
                ++g;
            }
    }
    // every box issued has landed before the CTA leaves (each slot's last box completes its
    // phase; a box already consumed has completed it long ago)
    for (uint32_t k = 0; k < (uint32_t)kABoxes && k < g; ++k) {
        const uint32_t gl = g - 1u - k;
        tc_wait(&a_full[gl % kABoxes], (gl / kABoxes) & 1u, no_abort);
    }
}

// ---- converter warps ---------------------------------------------------------------------------
// Thread = patch pixel = tensor-memory lane (warp c of the group owns lane quadrant c mod 4 and
// integrands 32 (c / 4) .. 32 (c / 4) + 31 of every slot): reads its part of its row of the box,
// converts it to centred f16 and stores 16 columns of the slot.
__device__ void tc_convert(const TcArgs &args, const TcUnit *utab, int nu, char *smem,
                           uint64_t *a_full, uint64_t *a_empty, uint64_t *full,
                           uint64_t *empty, uint32_t tmem, volatile int *abort_flag)
{
    const int cw = (threadIdx.x >> 5) - kConvWarp0;  // 0 .. kConvWarps - 1
    const int lane = threadIdx.x & 31;
    const int ct = 32 * (cw & 3) + lane;             // patch pixel, tensor-memory lane
    const int half = cw >> 2;
    const int lx = ct & 15, ly = ct >> 4;
    const uint32_t lane_base = (uint32_t)(ct & ~31) << 16;
    uint32_t gb = 0, gs = 0;
    bool ok = true;
    for (int ku = 0; ku < nu && ok; ++ku) {
        int pi;
        const Unit d = unit_at(utab, ku, pi);
        if (d.cnt <= 0) continue;
        const bool qin = d.x0 + lx < unit_w(d) && d.y0 + ly < unit_h(d);
        const int nbox = unit_row_bytes(d) >> 7;
        const bool wide = unit_count_bytes(d) == 2;
        // 1024 + k - (1024 + N/2) = k - N/2, exact
        const uint32_t hb = 0x6400u + (uint32_t)((d.t->nr & 0xFFFF) >> 1);
        const uint32_t bias = hb | (hb << 16);
        for (int n0 = 0; n0 < d.cnt && ok; n0 += kNB)
            for (int c = 0; c < nbox; ++c) {
                const uint32_t slot = gb % kABoxes, use = gb / kABoxes;
                if (!tc_wait_warp(&a_full[slot], use & 1u, abort_flag)) {
                    ok = false;
                    break;
                }
                const char *row = smem + kOffA + slot * kBoxBytes + ct * 128;
                const int nsub = wide ? 1 : 2;
                for (int sb = 0; sb < nsub; ++sb) {
                    const uint32_t as = gs % kStages, ause = gs / kStages;
                    if (!tc_wait_warp(&empty[as], (ause & 1u) ^ 1u, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    uint32_t o[16];
                    if (wide) {  // integrands 32 half .. of 64 of 16 bits: one f16x2 per word
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const uint4 x = *reinterpret_cast<const uint4 *>(
                                row + (((4 * half + j) ^ (ct & 7)) << 4));
                            o[4 * j + 0] = h2_sub(x.x | kH2Magic, bias);
                            o[4 * j + 1] = h2_sub(x.y | kH2Magic, bias);
                            o[4 * j + 2] = h2_sub(x.z | kH2Magic, bias);
                            o[4 * j + 3] = h2_sub(x.w | kH2Magic, bias);
                        }
                    } else {  // bytes 64 sb + 32 half .. + 31: two f16x2 per word
#pragma unroll
                        for (int j = 0; j < 2; ++j) {
                            const uint4 x = *reinterpret_cast<const uint4 *>(
                                row + (((4 * sb + 2 * half + j) ^ (ct & 7)) << 4));
                            bytes_to_h2(x.x, bias, o[8 * j + 0], o[8 * j + 1]);
                            bytes_to_h2(x.y, bias, o[8 * j + 2], o[8 * j + 3]);
                            bytes_to_h2(x.z, bias, o[8 * j + 4], o[8 * j + 5]);
                            bytes_to_h2(x.w, bias, o[8 * j + 6], o[8 * j + 7]);
                        }
                    }
                    if (!qin) {  // pixels outside a ragged tile: zero rows
#pragma unroll
                        for (int i = 0; i < 16; ++i) o[i] = 0u;
                    }
                    tc::tmem_st16(tmem + lane_base + kColA + 32u * as + 16u * half, o);
                    tc::fence_before_sync();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&full[as]);
                    ++gs;
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&a_empty[slot]);
                if (!ok) break;
                ++gb;
            }
    }
}

// ---- producer warps (B) ------------------------------------------------------------------------
// A stage holds up to kNB delta rows of 64 integrands, each row eight 16-byte pieces, copied by
// cp.async straight into the swizzled slots (piece j of row r in slot j ^ (r mod 8)).  Producer
// thread pt owns piece pt mod 8 of rows pt / 8 + kProdRowStep k: a warp copies four whole rows
// per instruction.  Each thread's copies of a stage arrive on the stage's barrier when they land
// (the barrier counts every producer thread), so up to kStages stages are in flight.  A warp
// issues cp.async at about 10 bytes per clock, so four warps share the stage.
// the first (first = true) or the next product of this CTA: its patch (table index) and first
// listed entry; false past the last one
__device__ __forceinline__ bool next_product(const TcArgs &args, const TcUnit *utab, int nu, int &ku,
                                             int &n0, Unit &d, int &pi, bool first)
{
    if (!first && n0 + kNB < d.cnt) {
        n0 += kNB;
        return true;
    }
    if (!first) ++ku;
    for (; ku < nu; ++ku) {
        d = unit_at(utab, ku, pi);
        if (d.cnt > 0) {
            n0 = 0;
            return true;
        }
    }
    return false;
}

// couple of each of this thread's rows of a product (-1: rows nn .. kNB - 1 stay unloaded, they
// feed columns the epilogue ignores)
__device__ __forceinline__ void product_rows(const Unit &d, int n0, int r0, int (&idx)[kBTasks])
{
    const int nn = d.cnt - n0 < kNB ? d.cnt - n0 : kNB;
    const int4 *list = d.t->list + n0;
#pragma unroll
    for (int k = 0; k < kBTasks; ++k) {
        const int row = r0 + kProdRowStep * k;
        idx[k] = row < nn ? (list[row].z >> 1) : -1;
    }
}

__device__ void tc_produce_b(const TcArgs &args, const TcUnit *utab, int nu, char *smem,
                             uint64_t *full, uint64_t *empty, volatile int *abort_flag)
{
    const int pt = threadIdx.x - kProdWarp0 * 32;
    // rows r0 + kProdRowStep k: r mod 8 = r0 mod 8, r / 8 = r0 / 8 + (kProdRowStep / 8) k
    const int piece = pt & 7, r0 = pt >> 3;
    const uint32_t dpos = tc::saddr(smem + kOffB) +
                          (uint32_t)((r0 >> 3) * 1024 + (r0 & 7) * 128 + ((piece ^ (r0 & 7)) << 4));
    uint32_t g = 0;
    bool ok = true;
    const uint64_t pol = policy_evict_last();
    int ku = 0, n0 = 0, pi = 0;
    Unit d{};
    bool have = next_product(args, utab, nu, ku, n0, d, pi, true);
    int idx[kBTasks];
    if (have) product_rows(d, n0, r0, idx);
    while (have && ok) {
        // the next product's rows are read while this one's stages are copied
        int ku2 = ku, n02 = n0, pi2 = pi;
        Unit d2 = d;
        const bool have2 = next_product(args, utab, nu, ku2, n02, d2, pi2, false);
        int idx2[kBTasks];
        if (have2) product_rows(d2, n02, r0, idx2);
        const int kst = unit_stages(d);
        const uint16_t *const del = d.t->delta + 8 * piece;
        const size_t dplane = (size_t)d.t->M << 6;  // f16 per stage
        for (int ks = 0; ks < kst; ++ks) {
            const uint32_t slot = g % kStages, use = g / kStages;
            if (!tc_wait_warp(&empty[slot], (use & 1u) ^ 1u, abort_flag)) {
                ok = false;
                break;
            }
            const uint32_t st = dpos + slot * kBStageBytes;
            const uint16_t *cd = del + (size_t)ks * dplane;
#pragma unroll
            for (int k = 0; k < kBTasks; ++k)
                if (idx[k] >= 0)
                    cp_async16(st + k * (kProdRowStep / 8) * 1024, cd + ((size_t)idx[k] << 6), pol);
            cp_async_arrive(&full[slot]);
            ++g;
        }
        ku = ku2;
        n0 = n02;
        pi = pi2;
        d = d2;
        have = have2;
#pragma unroll
        for (int k = 0; k < kBTasks; ++k) idx[k] = idx2[k];
    }
    cp_async_wait_all();  // nothing in flight when the CTA leaves
}

// ---- MMA warps ------------------------------------------------------------------------------
// Stage g of the CTA's sequence is issued by MMA warp g mod kMmaWarps, so that while one warp
// waits for its operands and commits its releases the others keep the tensor core's short
// issue queue filled.  The products are exact integers in f32 (no rounding), so the order in
// which the warps' products accumulate does not matter; every product accumulates onto an
// accumulator the epilogue has zeroed.  A product is complete when every MMA warp has committed
// it (acc_full counts kMmaWarps arrivals).
template <bool kRounds>
__device__ void tc_mma(const TcArgs &args, const TcUnit *utab, int nu, char *smem,
                       uint64_t *full, uint64_t *empty, uint64_t *acc_full, uint64_t *acc_empty,
                       uint64_t *done, uint32_t tmem, volatile int *abort_flag,
                       volatile int *no_abort)
{
    const int lane = threadIdx.x & 31;
    const int mw = (threadIdx.x >> 5) - kMmaWarp0;  // 0 .. kMmaWarps - 1
    const uint32_t sbase = tc::saddr(smem + kOffB);
    uint32_t g = 0, jb = 0;
    bool ok = true, issued = false;
    for (int ku = 0; ku < nu && ok; ++ku) {
        int pi;
        const Unit d = unit_at(utab, ku, pi);
        if (d.cnt <= 0) continue;
        const int kst = unit_stages(d), kper = kRounds ? d.t->kper : kst;
        for (int n0 = 0; n0 < d.cnt && ok; n0 += kNB)
        for (int s0 = 0; s0 < kst && ok; s0 += kper) {  // the product's accumulator rounds
            const int nn = d.cnt - n0 < kNB ? d.cnt - n0 : kNB;
            const int npad = (nn + 15) & ~15;
            const int sn = kst - s0 < kper ? kst - s0 : kper;
            const uint32_t buf = jb & 1u;
            // this warp's stages of the round: g .. g + sn - 1 with g' mod kMmaWarps == mw
            const uint32_t first = g + (uint32_t)((mw - (int)(g % kMmaWarps) + kMmaWarps) % kMmaWarps);
            if (first < g + (uint32_t)sn) {
                ok = tc_wait_warp(&acc_empty[buf], ((jb >> 1) & 1u) ^ 1u, abort_flag);
                if (!ok) break;
                tc::fence_after_sync();
            }
            const uint32_t dt = tmem + buf * kAccCols;
            const uint32_t idesc = tc::idesc_f16_f32(kTcM, npad);
            for (uint32_t gs = first; gs < g + (uint32_t)sn; gs += kMmaWarps) {
                const uint32_t as = gs % kStages;
                ok = tc_wait_warp(&full[as], (gs / kStages) & 1u, abort_flag);
                if (!ok) break;
                tc::fence_after_sync();
                if (lane == 0) {
                    // the delta rows were written by cp.async (generic proxy): make them
                    // visible to the tensor core's reads
                    tc::fence_async_smem();
                    tc::mma4_f16_ts_acc(dt, tmem + kColA + 32u * as,
                                        tc::sw128_desc(sbase + as * kBStageBytes, 0), idesc);
                    tc::mma_commit(&empty[as]);
                }
                __syncwarp();
                issued = true;
            }
            if (!ok) break;
            // this warp's part of the round is issued (possibly none of it)
            if (lane == 0) tc::mma_commit(&acc_full[buf]);
            __syncwarp();
            g += (uint32_t)sn;
            ++jb;
        }
    }
    // every product issued has completed before tensor memory is released
    if (issued) {
        if (lane == 0) tc::mma_commit(&done[mw]);
        __syncwarp();
        tc_wait(&done[mw], 0u, no_abort);
    }
}

// ---- epilogue warps ----------------------------------------------------------------------------
// Warp w reads lane quadrant w mod 4 (patch pixels 32 (w mod 4) ..) and columns 16 (w / 4) ..
// of every 32-column step.
template <bool kRounds>
__device__ void tc_epilogue(const TcArgs &args, const TcUnit *utab, int nu, char *smem,
                            uint64_t *acc_full, uint64_t *acc_empty, uint32_t tmem,
                            volatile int *abort_flag)
{
    const int et = threadIdx.x;  // 0 .. 255
    const int w = et >> 5, lane = et & 31;
    const int quad = w & 3, half = w >> 2;
    int32_t *dt = reinterpret_cast<int32_t *>(smem + kOffDt);  // [32][128] or [kNB][32]
    // per listed pixel, by product parity: (table offset, partner, slot, x | y << 16) and
    // (its patch-local x, y, the partner's patch pixel or -1, slot)
    int4 *colb = reinterpret_cast<int4 *>(smem + kOffCol);
    int4 *col1b = colb + 2 * kNB;
    int32_t *acc6 = reinterpret_cast<int32_t *>(smem + kOffAcc6);  // [kNB][kAccStride]
    int32_t *tab = reinterpret_cast<int32_t *>(smem + kOffTab);
    int8_t *tab2 = reinterpret_cast<int8_t *>(smem + kOffTab2);
    const int row = 32 * quad + lane;  // the patch pixel of this thread's accumulator lane
    const int lx = row & 15, ly = row >> 4;
    const uint32_t lane_base = (uint32_t)(32 * quad) << 16;
    uint32_t jb = 0;
    int cur = -1;
    int32_t *tc_cnt = nullptr;  // the current problem's list counts
    bool ok = true;
    for (int ku = 0; ku < nu && ok; ++ku) {
        int pi;
        const Unit d = unit_at(utab, ku, pi);
        if (d.cnt <= 0) continue;
        const int W = unit_w(d), H = unit_h(d), hw = W >> 1, hh = H >> 1;
        const int r = (d.t->nr >> 16) & 0xFF, r2 = r * r, ncls = d.t->nr >> 24;
        const bool fast = (d.t->flags & kUnitTable) != 0;
        const int tw = tab2_w(r);
        // compile-time path: radius 6 with the classes of the static stencil
        const bool colpath = (d.t->flags & kUnitStatic6) != 0;
        if (pi != cur) {  // class of each squared distance / offset of this problem
            const Problem &pb = args.probs[pi];
            epi_sync();
            for (int i = et; i < kTabMax; i += kEpiThreads) tab[i] = -1;
            epi_sync();
            if (et < ncls) tab[pb.d2[et]] = et;
            epi_sync();
            if (fast && !colpath) {
                const int dxm = tab2_dx(r), n2 = tw * (2 * tab2_dy(r) + 1);
                for (int i = et; i < n2; i += kEpiThreads) {
                    const int dx = i % tw - dxm, dy = i / tw - tab2_dy(r);
                    const int dd = dx * dx + dy * dy;
                    tab2[i] = (int8_t)(dd <= r2 ? tab[dd] : -1);
                }
                epi_sync();
            }
            cur = pi;
            tc_cnt = pb.tc_cnt;
        }
        const int qx = d.x0 + lx, qy = d.y0 + ly;
        const bool qin = qx < W && qy < H;
        const int qpix = qy * W + qx;
        // this lane's part of the 2-D table index (offsets from the patch centre)
        const int lt = (ly - kPH / 2 + tab2_dy(r)) * tw + (lx - kPW / 2 + tab2_dx(r));
        int32_t *const side = d.t->side;
        const int4 *list = d.t->list;
        for (int n0 = 0; n0 < d.cnt && ok; n0 += kNB)
        for (int rr = 0; rr < (kRounds ? (d.t->flags >> 8) : 1); ++rr) {  // one accumulator per
                                                                         // round, sums added
            const int nn = d.cnt - n0 < kNB ? d.cnt - n0 : kNB;
            const int npad = (nn + 15) & ~15;
            const uint32_t buf = jb & 1u;
            int4 *col = colb + (jb & 1u) * kNB, *col1 = col1b + (jb & 1u) * kNB;
            // the table paths reuse the scratch every product: the previous readers are done
            if (!colpath) epi_sync();
            for (int n = et; n < nn; n += kEpiThreads) {
                const int4 e = list[n0 + n];
                const int rx = (int)(int16_t)(e.w & 0xFFFF), ry = e.w >> 16;
                col[n] = make_int4(ry * tw + rx, e.y, e.z, (e.x % W) | ((e.x / W) << 16));
                const int ax = e.y % W - d.x0, ay = e.y / W - d.y0;
                const int plane = (ax >= 0 && ax < kPW && ay >= 0 && ay < kPH) ? ay * kPW + ax : -1;
                col1[n] = make_int4(rx + kPW / 2, ry + kPH / 2, plane, e.z);
            }
            if (!colpath) {
                for (int e = et; e < nn * 8; e += kEpiThreads)
                    reinterpret_cast<int4 *>(dt)[e] = make_int4(0, 0, 0, 0);
                epi_sync();
            }
            const bool wok = tc_wait(&acc_full[buf], (jb >> 1) & 1u, abort_flag);
            if (epi_any(!wok)) {
                ok = false;
                break;
            }
            tc::fence_after_sync();
            const int nch = (npad + 31) >> 5;
            for (int k = 0; k < nch; ++k) {
                const int c0 = 32 * k, cc = c0 + 16 * half;  // this warp's first column
                const bool have = cc < npad;                 // uniform per warp
                uint32_t v[16];
                if (have) {  // read, and leave zeros for the next product on this accumulator
                    const uint32_t ta = tmem + lane_base + buf * kAccCols + (uint32_t)cc;
                    tc::tmem_ld16(ta, v);
                    tc::tmem_zero16(ta);
                }
                if (k == nch - 1) {  // the accumulator is free once every lane has read it
                    tc::fence_before_sync();
                    mbar_arrive(&acc_empty[buf]);
                }
                if (colpath) {
                    int32_t *dtb = dt;
                    // the previous step's readers are done before the transpose is overwritten
                    // (a product's first step follows the previous product's final barrier)
                    if (k > 0) epi_sync();
                    if (have) {
#pragma unroll
                        for (int i = 0; i < 16; ++i)
                            dtb[(16 * half + i) * kTcM + row] =
                                __float2int_rn(__uint_as_float(v[i]));  // an exact integer
                    }
                    epi_sync();
                    const int n = c0 + lane;
                    if (n < nn) g6_warp(w, dtb + lane * kTcM, col1[n], lane, acc6 + n * kAccStride);
                } else if (have && qin && fast) {
                    // per column: the table lookup, then the class-sum update
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int n = cc + i;
                        if (n < nn) {
                            const int2 cinfo = *reinterpret_cast<const int2 *>(col + n);
                            const int c = tab2[lt - cinfo.x];
                            if (c >= 0 && qpix != cinfo.y)
                                atomicAdd(reinterpret_cast<int *>(dt) + n * 32 + c,
                                          __float2int_rn(__uint_as_float(v[i])));
                        }
                    }
                } else if (have && qin) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int n = cc + i;
                        if (n < nn) {
                            const int4 cinfo = col[n];
                            int dx = qx - (cinfo.w & 0xFFFF), dy = qy - (cinfo.w >> 16);
                            dx += dx < -hw ? W : 0;
                            dx -= dx > hw ? W : 0;
                            dy += dy < -hh ? H : 0;
                            dy -= dy > hh ? H : 0;
                            const int dd = dx * dx + dy * dy;  // |dx| <= W/2, |dy| <= H/2
                            if (dd <= r2) {
                                const int c = tab[dd];  // -1 for dd = 0 and empty classes
                                if (c >= 0 && qpix != cinfo.y)
                                    atomicAdd(reinterpret_cast<int *>(dt) + n * 32 + c,
                                              __float2int_rn(__uint_as_float(v[i])));
                            }
                        }
                    }
                }
            }
            if (colpath) {  // the product's class sums
                epi_sync();
                g6_flush(acc6, col1, nn, w, lane, side);
            } else {
                // warp w sends the class sums of columns w, w + 8, ...; lane = class
                epi_sync();
                for (int nb = w; nb < nn; nb += kEpiWarps * kFlushBatch) {
                    int val[kFlushBatch], slot[kFlushBatch];
#pragma unroll
                    for (int k = 0; k < kFlushBatch; ++k) {
                        const int n = nb + kEpiWarps * k;
                        slot[k] = n < nn ? col[n].z : 0;
                        val[k] = (n < nn && lane < ncls) ? dt[n * 32 + lane] : 0;
                        if (slot[k] & 1) val[k] = -val[k];  // the b side carries -delta
                    }
#pragma unroll
                    for (int k = 0; k < kFlushBatch; ++k)
                        if (val[k]) red_add_global(side + (size_t)slot[k] * kMaxClasses + lane, val[k]);
                }
                epi_sync();  // the scratch is free for the next product
            }
            ++jb;
        }
        if (!ok) break;
        if (et == 0) tc_cnt[d.pid] = 0;  // cleared for the next pass
    }
}

// kRounds: some problem of the launch sums its integrands in more than one accumulator round
template <bool kRounds>
__global__ void __launch_bounds__(kTcThreads, 1) k_tc_stencil(TcArgs args)
{
    extern __shared__ unsigned char smem_raw[];
    char *smem = reinterpret_cast<char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kOffBar);
    uint64_t *a_full = bars, *a_empty = a_full + kABoxes;
    uint64_t *full = a_empty + kABoxes, *empty = full + kStages;
    uint64_t *acc_full = empty + kStages, *acc_empty = acc_full + 2;
    uint64_t *done = acc_empty + 2;  // [kMmaWarps]
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(smem + kOffMisc);
    volatile int *s_abort = reinterpret_cast<volatile int *>(smem + kOffMisc + 4);
    volatile int *s_zero = reinterpret_cast<volatile int *>(smem + kOffMisc + 8);  // stays 0
    const int warp = threadIdx.x >> 5;
    // this CTA's patches: static part from the plan, listed pixels of this pass
    TcUnit *utab = reinterpret_cast<TcUnit *>(smem + kOffUnits);
    const int ufirst = args.unit_begin + blockIdx.x * args.per;
    const int ulast = min(ufirst + args.per, args.unit_begin + args.unit_count);
    const int nu = ulast > ufirst ? ulast - ufirst : 0;
    for (int k = threadIdx.x; k < nu; k += blockDim.x) {
        const int4 ui = args.units[ufirst + k];
        const Problem &pb = args.probs[ui.x];
        int c = 0;
        if (pb.ctr[0] < pb.ctr[1]) {
            c = pb.tc_cnt[ui.y];
            c = c < pb.tc_cap ? c : pb.tc_cap;
        }
        TcUnit t;
        t.pi = ui.x;
        t.pid = ui.y;
        t.cnt = c;
        t.xy = ui.z | (ui.w << 16);
        t.wh = pb.W | (pb.H << 16);
        t.geom = pb.row_bytes | (pb.count_bytes << 16);
        t.nr = pb.N | (pb.radius << 16) | (pb.n_cls << 24);
        t.M = pb.M;
        t.list = pb.tc_list + (size_t)ui.y * pb.tc_cap;
        t.delta = pb.tc_delta16;
        t.side = pb.side_cls;
        const bool fast = tab2_ok(pb.W, pb.H, pb.radius);
        const bool st6 = fast && pb.radius == 6 && pb.n_cls == kCls6 &&
                         classes_match6(pb.d2, std::make_integer_sequence<int, kCls6>{});
        t.kper = tc_round_stages(pb.N, tc_stages(pb));
        t.flags = (fast ? kUnitTable : 0) | (st6 ? kUnitStatic6 : 0) |
                  (((tc_stages(pb) + t.kper - 1) / t.kper) << 8);
        utab[k] = t;
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < kABoxes; ++i) {
            mbar_init(&a_full[i], 1);
            mbar_init(&a_empty[i], kConvWarps);
        }
        for (int i = 0; i < kStages; ++i) {  // a stage is full when both operands are in
            mbar_init(&full[i], kConvWarps + kProdThreads);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&acc_full[i], kMmaWarps);
            mbar_init(&acc_empty[i], kEpiThreads);
        }
        for (int i = 0; i < kMmaWarps; ++i) mbar_init(&done[i], 1);
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
    // both accumulators start at zero (every product accumulates onto them; the epilogue
    // zeroes what it reads)
    if (warp < kEpiWarps) {
        const uint32_t q = (uint32_t)(32 * (warp & 3)) << 16;
        for (uint32_t c = 16u * (warp >> 2); c < 2 * kAccCols; c += 32u) tc::tmem_zero16(tmem + q + c);
        tc::fence_before_sync();
    }
    __syncthreads();
    tc::fence_after_sync();
    if (warp < kConvWarp0)
        tc_epilogue<kRounds>(args, utab, nu, smem, acc_full, acc_empty, tmem, s_abort);
    else if (warp < kProdWarp0)
        tc_convert(args, utab, nu, smem, a_full, a_empty, full, empty, tmem, s_abort);
    else if (warp < kLoadWarp)
        tc_produce_b(args, utab, nu, smem, full, empty, s_abort);
    else if (warp == kLoadWarp) {
        if ((threadIdx.x & 31) == 0)
            tc_load_a(args, utab, nu, smem, a_full, a_empty, s_abort, s_zero);
    } else
        tc_mma<kRounds>(args, utab, nu, smem, full, empty, acc_full, acc_empty, done, tmem, s_abort,
                        s_zero);
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

// patch i met at |offset| ad: a new entry, or a smaller offset for a known one (fully unrolled,
// so the small arrays stay in registers)
__device__ __forceinline__ void note_patch(int (&idx)[kMaxMet], int (&dist)[kMaxMet], int &n,
                                           int i, int ad)
{
    bool found = false;
#pragma unroll
    for (int k = 0; k < kMaxMet; ++k)
        if (k < n && idx[k] == i) {
            dist[k] = ad < dist[k] ? ad : dist[k];
            found = true;
        }
    if (!found && n < kMaxMet) {
#pragma unroll
        for (int k = 0; k < kMaxMet; ++k)
            if (k == n) {
                idx[k] = i;
                dist[k] = ad;
            }
        ++n;
    }
}
__device__ __forceinline__ int pick(const int (&a)[kMaxMet], int i)
{
    int v = a[0];
#pragma unroll
    for (int k = 1; k < kMaxMet; ++k) v = i == k ? a[k] : v;
    return v;
}

// Distinct patches (of size ps along an axis of n pixels) met by the window [c - r, c + r],
// torus-wrapped (r < n), with the smallest |offset| reaching each.  The window is walked in runs
// of pixels of one patch (at most four for r <= 8); a run can meet a patch met before when the
// window wraps on a narrow torus, so every run is merged into the list.
__device__ __forceinline__ void axis_patches(int c, int r, int n, int ps, int (&idx)[kMaxMet],
                                             int (&dist)[kMaxMet], int &cnt)
{
    const int total = 2 * r + 1;
    int x = wrap_add(c, -r, n), done = 0;  // window offsets covered so far: done - r ..
    while (done < total) {
        const int pc = x / ps;
        const int cend = (pc + 1) * ps < n ? (pc + 1) * ps : n;
        const int len = cend - x < total - done ? cend - x : total - done;
        const int d0 = done - r, d1 = done + len - 1 - r;  // offsets of the run
        const int a0 = d0 < 0 ? -d0 : d0, a1 = d1 < 0 ? -d1 : d1;
        note_patch(idx, dist, cnt, pc, (d0 <= 0 && d1 >= 0) ? 0 : (a0 < a1 ? a0 : a1));
        done += len;
        x += len;
        x -= x >= n ? n : 0;
    }
}

// One warp per couple: the couple's class sums are cleared, its f16 delta row k_b - k_a is
// written for every stage of 64 integrands, and each of its two pixels is appended to the lists
// of the patches within the radius of it (lanes 0-15: pixel a, 16-31: pixel b, one patch per
// lane).
// eight CTAs of 256 threads per SM (32 registers): occupancy over the few spills it costs
__global__ void __launch_bounds__(kListThreads, 8) k_tc_lists(const Problem *probs)
{
    const Problem &pb = probs[blockIdx.y];
    const long long s = pb.ctr[0];
    if (s >= pb.ctr[1]) return;
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.x * (kListThreads / 32) + (threadIdx.x >> 5);
    if (j >= pb.M) return;
    const uint32_t xs = pass_xor(pb, (uint32_t)s);
    const int a = (int)((uint32_t)pb.perm[2 * j] ^ xs);
    const int b = (int)((uint32_t)pb.perm[2 * j + 1] ^ xs);
    if (a >= pb.P || b >= pb.P) return;
    if (lane < 2 * kMaxClasses / 4)
        reinterpret_cast<int4 *>(pb.side_cls + (size_t)j * 2 * kMaxClasses)[lane] =
            make_int4(0, 0, 0, 0);
    const int kst = tc_stages(pb);
    // two steps (v, v + 32) per lane and iteration, both steps' loads issued before either
    // step's stores
    if (pb.count_bytes == 1) {
        // 16 integrands (two f16 pieces of one stage) per lane and step
        const int nv = kst * 4;
        for (int v = lane; v < nv; v += 64) {
            const bool two = v + 32 < nv;
            uint4 ka[2], kb[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int e0 = (v + 32 * h) * 16;  // first integrand
                const size_t off = (((size_t)(e0 >> 7) * pb.P) << 7) + (e0 & 127);
                ka[h] = kb[h] = make_uint4(0u, 0u, 0u, 0u);
                if (h == 0 || two) {
                    ka[h] = *reinterpret_cast<const uint4 *>(pb.counts + ((size_t)a << 7) + off);
                    kb[h] = *reinterpret_cast<const uint4 *>(pb.counts + ((size_t)b << 7) + off);
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int vh = v + 32 * h;
                if (h == 1 && !two) break;
                uint4 o0, o1;
                bytes_sub_h2(kb[h].x, ka[h].x, o0.x, o0.y);
                bytes_sub_h2(kb[h].y, ka[h].y, o0.z, o0.w);
                bytes_sub_h2(kb[h].z, ka[h].z, o1.x, o1.y);
                bytes_sub_h2(kb[h].w, ka[h].w, o1.z, o1.w);
                uint4 *dst = reinterpret_cast<uint4 *>(pb.tc_delta16 +
                                                       (((size_t)(vh >> 2) * pb.M + j) << 6) +
                                                       (vh & 3) * 16);
                dst[0] = o0;
                dst[1] = o1;
            }
        }
    } else {
        // 16-bit counts (below 1024): 8 integrands (one f16 piece) per lane and step; a stage
        // of 64 integrands is one 128-byte chunk
        const int nv = kst * 8;
        for (int v = lane; v < nv; v += 64) {
            const bool two = v + 32 < nv;
            uint4 ka[2], kb[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int e0 = (v + 32 * h) * 8;
                const size_t off = (((size_t)(e0 >> 6) * pb.P) << 7) + (e0 & 63) * 2;
                ka[h] = kb[h] = make_uint4(0u, 0u, 0u, 0u);
                if (h == 0 || two) {
                    ka[h] = *reinterpret_cast<const uint4 *>(pb.counts + ((size_t)a << 7) + off);
                    kb[h] = *reinterpret_cast<const uint4 *>(pb.counts + ((size_t)b << 7) + off);
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int e0 = (v + 32 * h) * 8;
                if (h == 1 && !two) break;
                uint4 o;
                o.x = h2_sub(kb[h].x | kH2Magic, ka[h].x | kH2Magic);
                o.y = h2_sub(kb[h].y | kH2Magic, ka[h].y | kH2Magic);
                o.z = h2_sub(kb[h].z | kH2Magic, ka[h].z | kH2Magic);
                o.w = h2_sub(kb[h].w | kH2Magic, ka[h].w | kH2Magic);
                *reinterpret_cast<uint4 *>(pb.tc_delta16 + (((size_t)(e0 >> 6) * pb.M + j) << 6) +
                                           (e0 & 63)) = o;
            }
        }
    }
    // lanes 0..15 list pixel a, lanes 16..31 pixel b, one patch each, all atomics in parallel
    const int side = lane >> 4, k = lane & 15;
    const int r = pb.radius, r2 = r * r;
    const int p = side ? b : a, px = p % pb.W, py = p / pb.W;
    // distinct patch columns (rows) met by x in [px - r, px + r] (y likewise), torus-wrapped,
    // with the smallest |offset| that reaches each
    int xi[kMaxMet], xd[kMaxMet], yi[kMaxMet], yd[kMaxMet], nx = 0, ny = 0;
    axis_patches(px, r, pb.W, kPW, xi, xd, nx);
    axis_patches(py, r, pb.H, kPH, yi, yd, ny);
    // at most 3 x 4 patches for radius <= 8; the loop covers any count
    for (int kk = k; kk < nx * ny; kk += 16) {
        const int u = kk / ny, w = kk - (kk / ny) * ny;  // this lane's patch
        const int xdu = pick(xd, u), ydw = pick(yd, w);
        if (xdu * xdu + ydw * ydw <= r2) {  // in reach
            const int xiu = pick(xi, u), yiw = pick(yi, w);
            const int pid = yiw * pb.tc_npx + xiu;
            const int pos = atomicAdd(pb.tc_cnt + pid, 1);
            // min-image offset of p from the patch centre
            int rx = px - (xiu * kPW + kPW / 2), ry = py - (yiw * kPH + kPH / 2);
            rx -= rx > (pb.W >> 1) ? pb.W : 0;
            rx += rx < -(pb.W >> 1) ? pb.W : 0;
            ry -= ry > (pb.H >> 1) ? pb.H : 0;
            ry += ry < -(pb.H >> 1) ? pb.H : 0;
            if (pos < pb.tc_cap)
                pb.tc_list[(size_t)pid * pb.tc_cap + pos] =
                    make_int4(p, side ? a : b, 2 * j + side, (rx & 0xFFFF) | (ry << 16));
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
            // the two sides' class sums: two 128-byte rows, read as 16-byte vectors
            const int4 *ca = reinterpret_cast<const int4 *>(pb.side_cls +
                                                            (size_t)j * 2 * kMaxClasses);
            const int4 *cb = ca + kMaxClasses / 4;
            int A[kMaxClasses];
#pragma unroll
            for (int v = 0; v < kMaxClasses / 4; ++v) {
                const int4 x = ca[v], y = cb[v];
                A[4 * v + 0] = x.x + y.x;
                A[4 * v + 1] = x.y + y.y;
                A[4 * v + 2] = x.z + y.z;
                A[4 * v + 3] = x.w + y.w;
            }
#pragma unroll
            for (int c = 0; c < kMaxClasses; ++c) A[c] = c < pb.n_cls ? A[c] : 0;
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

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link against libcuda)
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

}  // namespace

bool tc_supported(const Problem &h)
{
    // counts below 1024 (f16 read as 1024 + k); accumulator rounds of at least one stage exact
    // in f32 (64 N^2 <= 2^25, N <= 724) and class sums within int32 (12 T N^2 < 2^31)
    const bool counts_ok = h.count_bytes == 1 || (h.count_bytes == 2 && h.N <= 512);
    const bool exact = (long long)h.T * h.N * h.N <= (1ll << 27);
    return counts_ok && exact && h.radius >= 1 && h.radius <= 8 && h.W >= 2 * h.radius + 1 &&
           h.H >= 2 * h.radius + 1 && h.n_cls <= kMaxClasses && h.row_bytes % 128 == 0;
}

int tc_units_per_problem(const Problem &h) { return h.tc_npx * h.tc_npy; }

bool tc_rounds(const Problem &h) { return tc_round_stages(h.N, tc_stages(h)) < tc_stages(h); }

size_t tc_delta_bytes(const Problem &h) { return (size_t)h.M * tc_stages(h) * 64 * 2; }

int tc_tensor_map_bytes() { return kTensorMapBytes; }

// the count planes [chunk][y][x][128 bytes] as a 4-D tensor; one box is a patch (16 x 8 pixels)
// of one chunk, 128-byte swizzle, zero outside the tile
cudaError_t encode_tc_tensor_map(const Problem &h, void *out)
{
    static const EncodeTiledFn fn = []() -> EncodeTiledFn {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000,
                                             cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<EncodeTiledFn>(ptr);
    }();
    if (!fn) {
        cudaGetLastError();
        return cudaErrorNotSupported;
    }
    const cuuint64_t dims[4] = {128u, (cuuint64_t)h.W, (cuuint64_t)h.H,
                                (cuuint64_t)(h.row_bytes / 128)};
    const cuuint64_t strides[3] = {128u, (cuuint64_t)h.W * 128u, (cuuint64_t)h.P * 128u};
    const cuuint32_t box[4] = {128u, (cuuint32_t)kPW, (cuuint32_t)kPH, 1u};
    const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
    const CUresult r =
        fn(static_cast<CUtensorMap *>(out), CU_TENSOR_MAP_DATA_TYPE_UINT8, 4, (void *)h.counts,
           dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t prepare_tc()
{
    cudaError_t e = cudaFuncSetAttribute(k_tc_stencil<false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_tc_stencil<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kSmemBytes);
    return e;
}

cudaError_t launch_tc_sweep(const TcLaunch &tl, cudaStream_t st, KernelTimer *tm)
{
    const dim3 gl((tl.max_M + kListThreads - 1) / kListThreads, tl.n_prob);
    const dim3 gw((tl.max_M + kListThreads / 32 - 1) / (kListThreads / 32), tl.n_prob);
    const bool timed = tm && tm->enabled, all = timed && tm->detail;
    if (all) tm->begin(kKTcLists, st);
    k_tc_lists<<<gw, kListThreads, 0, st>>>(tl.dprob);
    if (all) tm->end(st);
    if (tl.total_units > 0) {
        // each CTA takes a contiguous run of at most kUnitTab patches; a pass with more
        // patches than the SMs hold that way is split over launches of equal size
        const int nl = (tl.total_units + kUnitTab * tl.sms - 1) / (kUnitTab * tl.sms);
        const int per = (tl.total_units + nl * tl.sms - 1) / (nl * tl.sms);
        if (timed) tm->begin(kKTcStencil, st);
        for (int b0 = 0; b0 < tl.total_units; b0 += per * tl.sms) {
            const int cnt = tl.total_units - b0 < per * tl.sms ? tl.total_units - b0 : per * tl.sms;
            const TcArgs a{tl.dprob, tl.n_prob, tl.units, b0, cnt, per, tl.tmaps};
            if (tl.rounds)
                k_tc_stencil<true><<<(cnt + per - 1) / per, kTcThreads, kSmemBytes, st>>>(a);
            else
                k_tc_stencil<false><<<(cnt + per - 1) / per, kTcThreads, kSmemBytes, st>>>(a);
            note_launches(1);
        }
        if (timed) tm->end(st);
    }
    if (all) tm->begin(kKTcFinalize, st);
    k_tc_finalize<<<gl, kListThreads, 0, st>>>(tl.dprob);
    if (all) tm->end(st);
    note_launches(2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_resolve_commit(SweepLaunch{tl.dprob, tl.n_prob, tl.max_M, 1}, st, tm);
}

}  // namespace bn
