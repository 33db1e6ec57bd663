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
// radius of it (the patch's list, at most 160 per product), accumulating over all T integrands
// in tensor memory; about a fifth of the entries lie inside the radius and are kept.  The f16
// operands are exact (counts <= 64, |delta| <= 64) and the f32 sums stay within 2^24
// (T N^2 <= 2^24 for 8-bit counts), so every kept entry is an exact integer.
//
// A pass:
//   k_tc_lists     one warp per couple of the pass (as in the plain schedule): its class sums
//                  cleared, its f16 delta row k_b - k_a written for every stage, and each of its
//                  pixels appended to the list of every patch within the radius of it
//   k_tc_stencil   one CTA per SM over the patches, warp-specialised:
//                    9 producer warps   cp.async of whole 128-byte rows (four per warp
//                                       instruction) of the f16 count copy (A) and of the
//                                       delta rows (B) straight into the 128-byte swizzled
//                                       K-major layout; stages of 64 integrands
//                    1 MMA warp         four tcgen05.mma (K = 16 each) per stage
//                    4 epilogue warps   tensor memory -> registers; for radius 6 a transpose
//                                       of 32 columns through shared memory, each warp summing
//                                       a quarter of the stencil offsets per listed pixel with
//                                       compile-time classes; other radii a 2-D class table per
//                                       entry; class sums to global memory (integer reductions)
//                  five stages in a ring, two accumulator buffers in tensor memory
//   k_tc_finalize  change of Eq. 1 from the class sums, flags and pixel claims
//   then the resolve and commit kernels of the plain schedule (the commit also swaps the f16
//   copy, which k_tc_refresh rebuilds from the counts at the start of every run).
// Every wait is bounded; a wait that runs out raises the problems' error word and the CTA
// drains its copies and products, frees its tensor memory and returns.
#include <utility>

#include "bn_launch.h"
#include "bn_tcgen05.cuh"

namespace bn {
namespace {

constexpr int kPW = 16, kPH = 8, kTcM = kPW * kPH;  // patch: M = 128 pixels
constexpr int kNB = 160;                             // listed pixels per product (N)
constexpr int kStages = 5;                           // ring of 64-integrand stages
constexpr int kLook = 3;                             // stages in flight per producer thread
constexpr int kAStage = kTcM * 128;                  // 16 KB: 128 rows x 64 f16
constexpr int kBStage = kNB * 128;                   // 20 KB: 160 rows x 64 f16
constexpr int kStageBytes = kAStage + kBStage;
constexpr int kEpiWarps = 4, kProdWarps = (kTcM + kNB) / 32;  // eight pieces per thread
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kProdThreads = kProdWarps * 32;
constexpr int kMmaWarp = kEpiWarps + kProdWarps;
constexpr int kTcThreads = (kMmaWarp + 1) * 32;      // 448
constexpr uint32_t kTmemCols = 512, kTmemBuf = 256;  // two accumulator buffers
constexpr int kTabMax = 65;                          // squared distances 0..64 (radius <= 8)
constexpr long long kSpin = 1ll << 31;               // ~1 s at 2 GHz
constexpr unsigned long long kErrTc = 3ull;
constexpr int kFlushBatch = 5;                       // class-sum rows sent per batch

// shared memory layout (offsets from a 1024-byte aligned base)
// epilogue scratch: int32 [kNB][32] class sums (lane-per-pixel paths), or a 32-column transpose
// of the accumulators, float [32][128], and per-warp partial class sums, int32 [4][32][33]
// (column-per-thread path)
constexpr int kOffAcc = kStages * kStageBytes;
constexpr int kOffPart = kOffAcc + 32 * kTcM * 4;
constexpr int kEpiScratch = kNB * 32 * 4 > 32 * kTcM * 4 + 4 * 32 * 33 * 4
                                ? kNB * 32 * 4
                                : 32 * kTcM * 4 + 4 * 32 * 33 * 4;
constexpr int kOffCol = kOffAcc + kEpiScratch;        // int4 [2][kNB] per listed pixel
constexpr int kOffTab = kOffCol + 2 * kNB * 16;       // int32 [80] class of a squared distance
constexpr int kOffTab2 = kOffTab + 80 * 4;            // int8 [2-D offset] class (fast path)
constexpr int kTab2Max = 1664;                        // (2 (16 + 8) + 1) x (2 (8 + 8) + 1)
constexpr int kOffBar = kOffTab2 + kTab2Max;          // mbarriers
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
// integer add to global memory without a return value
__device__ __forceinline__ void red_add_global(int32_t *p, int v)
{
    // no compiler memory barrier: nothing in the kernel reads these sums
    asm volatile("red.global.add.s32 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "r"(v));
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

// four bytes -> two f16x2 (bytes 0,1 and 2,3); the bytes are read as 1024 + byte and 1024 is
// subtracted, so the values are exact
__device__ __forceinline__ void bytes_to_h2(uint32_t x, uint32_t bias2, uint32_t &lo, uint32_t &hi)
{
    const uint32_t a = __byte_perm(x, 0x64646464u, 0x4140);
    const uint32_t b = __byte_perm(x, 0x64646464u, 0x4342);
    asm("sub.f16x2 %0, %1, %2;" : "=r"(lo) : "r"(a), "r"(bias2));
    asm("sub.f16x2 %0, %1, %2;" : "=r"(hi) : "r"(b), "r"(bias2));
}
constexpr uint32_t kBiasCount = 0x64006400u;  // f16x2 (1024, 1024)
// four byte differences a - b -> two f16x2: both read as 1024 + byte, then subtracted
__device__ __forceinline__ void bytes_sub_h2(uint32_t a, uint32_t b, uint32_t &lo, uint32_t &hi)
{
    const uint32_t a0 = __byte_perm(a, 0x64646464u, 0x4140);
    const uint32_t a1 = __byte_perm(a, 0x64646464u, 0x4342);
    const uint32_t b0 = __byte_perm(b, 0x64646464u, 0x4140);
    const uint32_t b1 = __byte_perm(b, 0x64646464u, 0x4342);
    asm("sub.f16x2 %0, %1, %2;" : "=r"(lo) : "r"(a0), "r"(b0));
    asm("sub.f16x2 %0, %1, %2;" : "=r"(hi) : "r"(a1), "r"(b1));
}

// The unit decode shared by the three roles: the same global sequence of patches and of
// products (jobs) on every role, from values that do not change during the launch.
struct Unit {
    const Problem *pb;
    int pid, cnt, x0, y0;
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
    return d;
}

// 2-D class table of the epilogue's fast path: offsets (dx, dy) from a proposed pixel to a patch
// pixel, |dx| <= 16 + r, |dy| <= 8 + r, row-major with row length 2 (16 + r) + 1
__host__ __device__ __forceinline__ int tab2_dx(int r) { return 16 + r; }
__host__ __device__ __forceinline__ int tab2_dy(int r) { return 8 + r; }
__host__ __device__ __forceinline__ int tab2_w(int r) { return 2 * (16 + r) + 1; }
// the fast path holds when the torus is wide enough that a proposed pixel's offset from the patch
// centre, taken as the min-image, is its true offset (below half a side): W > 2 (8 + r),
// H > 2 (4 + r)
__host__ __device__ __forceinline__ bool tab2_ok(int W, int H, int r)
{
    return W > 2 * (8 + r) && H > 2 * (4 + r);
}

// ---- compile-time stencil of radius 6: offsets with 0 < dx^2 + dy^2 <= 36, by class ----------
struct Stencil6 {
    int n = 0, ncls = 0;
    int dx[169] = {}, dy[169] = {}, cls[169] = {}, d2[32] = {};
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
                        ++n;
                        any = true;
                    }
            if (any) d2[ncls++] = dd;
        }
    }
};
constexpr Stencil6 kSt6{};
constexpr int kCls6 = 18, kOffPerWarp = 28;
static_assert(kSt6.n == 4 * kOffPerWarp && kSt6.ncls == kCls6, "radius-6 stencil");

// one offset of the radius-6 stencil: the accumulator row of patch pixel p + offset, if that
// pixel is in the patch and is not the partner, added to its class sum
template <int O>
__device__ __forceinline__ void stencil_add(const float *dtc, int plx, int ply, int plane,
                                            int lane, int (&a)[kCls6])
{
    constexpr int dx = kSt6.dx[O], dy = kSt6.dy[O], c = kSt6.cls[O];
    const int lx = plx + dx, ly = ply + dy;
    const int q = ly * kPW + lx;
    const bool in = (unsigned)lx < (unsigned)kPW && (unsigned)ly < (unsigned)kPH && q != plane;
    // unconditional load; a lane outside the patch reads its own bank (row lane of its column)
    const float x = dtc[in ? q : lane];
    a[c] += in ? __float2int_rn(x) : 0;  // an exact integer held in f32
}
template <int Q, int... I>
__device__ __forceinline__ void stencil_quarter(const float *dtc, int plx, int ply, int plane,
                                                int lane, int (&a)[kCls6],
                                                std::integer_sequence<int, I...>)
{
    (stencil_add<Q * kOffPerWarp + I>(dtc, plx, ply, plane, lane, a), ...);
}
// warp w's quarter of the stencil offsets
__device__ __forceinline__ void stencil_warp(int w, const float *dtc, int4 c1, int lane,
                                             int (&a)[kCls6])
{
    using Seq = std::make_integer_sequence<int, kOffPerWarp>;
    switch (w) {
    case 0: stencil_quarter<0>(dtc, c1.x, c1.y, c1.z, lane, a, Seq{}); break;
    case 1: stencil_quarter<1>(dtc, c1.x, c1.y, c1.z, lane, a, Seq{}); break;
    case 2: stencil_quarter<2>(dtc, c1.x, c1.y, c1.z, lane, a, Seq{}); break;
    default: stencil_quarter<3>(dtc, c1.x, c1.y, c1.z, lane, a, Seq{}); break;
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

// ---- producer warps -----------------------------------------------------------------------
// A stage holds 128 A rows (the patch pixels' f16 counts) and up to kNB B rows (the listed
// couples' f16 deltas) of 64 integrands, each row eight 16-byte pieces, copied by cp.async
// straight into the swizzled slots (piece j of row r in slot j ^ (r mod 8)).  Producer thread pt
// owns the pieces pt + kProdThreads k, k < kTasks: a warp copies four whole 128-byte rows per
// instruction.  A rows of pixels outside a ragged tile are written as zeros.
constexpr int kTasks = 8;
static_assert(kTasks * kProdThreads == 8 * (kTcM + kNB), "one piece per task");
static_assert(kProdThreads % 8 == 0, "the piece index is the same for all of a thread's tasks");

// row kinds of a producer task
enum : int { kRowNone = 0, kRowCount = 1, kRowDelta = 2, kRowZero = 3 };

// make this thread's copies (and zero stores) of stage gi visible to the tensor core, then one
// arrival per warp
__device__ __forceinline__ void publish(char *smem, uint64_t *full, uint32_t gi, uint32_t kinds,
                                        const uint32_t (&roff)[kTasks], int piece)
{
    char *st = smem + (gi % kStages) * kStageBytes;
#pragma unroll
    for (int k = 0; k < kTasks; ++k)
        if (((kinds >> (2 * k)) & 3u) == (uint32_t)kRowZero)
            reinterpret_cast<uint4 *>(st + roff[k])[piece ^ ((roff[k] >> 7) & 7u)] =
                make_uint4(0u, 0u, 0u, 0u);
    tc::fence_async_smem();
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(&full[gi % kStages]);
}

__device__ void tc_produce(const TcArgs &args, char *smem, uint64_t *full, uint64_t *empty,
                           volatile int *abort_flag)
{
    const int pt = threadIdx.x - kEpiThreads;
    const int piece = pt & 7;
    constexpr int kRowStep = kProdThreads / 8;  // rows between a thread's tasks
    uint32_t roff[kTasks];
#pragma unroll
    for (int k = 0; k < kTasks; ++k) {
        const int row = (pt >> 3) + kRowStep * k, n = row - kTcM;
        roff[k] = row < kTcM ? (uint32_t)((row >> 3) * 1024 + (row & 7) * 128)
                             : (uint32_t)(kAStage + (n >> 3) * 1024 + (n & 7) * 128);
    }
    const uint32_t sbase = tc::saddr(smem);
    uint32_t kh[kLook];  // packed task kinds of the stages 1 .. kLook back
#pragma unroll
    for (int b = 0; b < kLook; ++b) kh[b] = 0u;
    uint32_t g = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < args.total_units && ok; u += gridDim.x) {
        int pi;
        const Unit d = decode_unit(args, u, pi);
        if (d.cnt <= 0) continue;
        const Problem &pb = *d.pb;
        const int nks = pb.row_bytes >> 6;
        const uint16_t *const cnt16 = pb.tc_counts16 + 8 * piece;
        const uint16_t *const del16 = pb.tc_delta16 + 8 * piece;
        const size_t cplane = (size_t)pb.P << 6, dplane = (size_t)pb.M << 6;  // f16 per stage
        const int4 *list = pb.tc_list + (size_t)d.pid * pb.tc_cap;
        for (int n0 = 0; n0 < d.cnt && ok; n0 += kNB) {
            const int nn = d.cnt - n0 < kNB ? d.cnt - n0 : kNB;
            uint32_t kinds = 0u;
            int idx[kTasks];  // pixel (A) or couple (B) of each task
#pragma unroll
            for (int k = 0; k < kTasks; ++k) {
                int kind = kRowNone;
                idx[k] = 0;
                const int row = (pt >> 3) + kRowStep * k;
                if (row < kTcM) {
                    const int qx = d.x0 + (row & 15), qy = d.y0 + (row >> 4);
                    if (qx < pb.W && qy < pb.H) {
                        kind = kRowCount;
                        idx[k] = qy * pb.W + qx;
                    } else {
                        kind = kRowZero;
                    }
                } else if (row - kTcM < nn) {  // rows nn .. npad - 1 feed ignored columns
                    kind = kRowDelta;
                    idx[k] = list[n0 + row - kTcM].z >> 1;  // couple of the listed slot
                }
                kinds |= (uint32_t)kind << (2 * k);
            }
            for (int ks = 0; ks < nks; ++ks) {
                const uint32_t slot = g % kStages, use = g / kStages;
                if (!tc_wait(&empty[slot], (use & 1u) ^ 1u, abort_flag)) {
                    ok = false;
                    break;
                }
                const uint32_t st = sbase + slot * kStageBytes;
                const uint16_t *ca = cnt16 + (size_t)ks * cplane;
                const uint16_t *cd = del16 + (size_t)ks * dplane;
#pragma unroll
                for (int k = 0; k < kTasks; ++k) {
                    const uint32_t kind = (kinds >> (2 * k)) & 3u;
                    const uint32_t dst = st + roff[k] + ((piece ^ ((roff[k] >> 7) & 7u)) << 4);
                    if (kind == (uint32_t)kRowCount) cp_async16(dst, ca + ((size_t)idx[k] << 6));
                    if (kind == (uint32_t)kRowDelta) cp_async16(dst, cd + ((size_t)idx[k] << 6));
                }
                cp_async_commit();
                if (g >= (uint32_t)kLook) {
                    cp_async_wait<kLook>();
                    publish(smem, full, g - kLook, kh[kLook - 1], roff, piece);
                }
#pragma unroll
                for (int b = kLook - 1; b > 0; --b) kh[b] = kh[b - 1];
                kh[0] = kinds;
                ++g;
            }
        }
    }
    cp_async_wait<0>();
    if (ok) {  // the last kLook stages, oldest first
#pragma unroll
        for (int b = kLook - 1; b >= 0; --b)
            if (g >= (uint32_t)(b + 1))
                publish(smem, full, g - (uint32_t)(b + 1), kh[b], roff, piece);
    }
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
    float *dt = reinterpret_cast<float *>(smem + kOffAcc);         // [32][128], column path
    int32_t *part = reinterpret_cast<int32_t *>(smem + kOffPart);  // [4][32][33], column path
    // per listed pixel: (table offset, partner, slot, x | y << 16) and, for the column path,
    // (its patch-local x, y, the partner's patch pixel or -1)
    int4 *col = reinterpret_cast<int4 *>(smem + kOffCol);
    int4 *col1 = col + kNB;
    int32_t *tab = reinterpret_cast<int32_t *>(smem + kOffTab);
    int8_t *tab2 = reinterpret_cast<int8_t *>(smem + kOffTab2);
    uint32_t jb = 0;
    int cur = -1;
    bool ok = true;
    for (int u = blockIdx.x; u < args.total_units && ok; u += gridDim.x) {
        int pi;
        const Unit d = decode_unit(args, u, pi);
        const Problem &pb = *d.pb;
        const int W = pb.W, H = pb.H, hw = W >> 1, hh = H >> 1;
        const int r = pb.radius, r2 = r * r, ncls = pb.n_cls;
        const bool fast = tab2_ok(W, H, r);
        const int tw = tab2_w(r);
        // column-per-thread path: radius 6 with the classes of the static stencil
        const bool colpath = fast && r == 6 && ncls == kCls6 &&
                             classes_match6(pb.d2, std::make_integer_sequence<int, kCls6>{});
        if (d.cnt > 0 && pi != cur) {  // class of each squared distance / offset of this problem
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
        }
        const int lx = et & 15, ly = et >> 4;
        const int qx = d.x0 + lx, qy = d.y0 + ly;
        const bool qin = qx < W && qy < H;
        const int qpix = qy * W + qx;
        // this lane's part of the 2-D table index (offsets from the patch centre)
        const int lt = (ly - kPH / 2 + tab2_dy(r)) * tw + (lx - kPW / 2 + tab2_dx(r));
        int32_t *const side = pb.side_cls;
        const int4 *list = pb.tc_list + (size_t)d.pid * pb.tc_cap;
        for (int n0 = 0; n0 < d.cnt; n0 += kNB) {
            const int nn = d.cnt - n0 < kNB ? d.cnt - n0 : kNB;
            const int npad = (nn + 15) & ~15;
            const uint32_t buf = jb & 1u;
            for (int n = et; n < nn; n += kEpiThreads) {
                const int4 e = list[n0 + n];
                const int rx = (int)(int16_t)(e.w & 0xFFFF), ry = e.w >> 16;
                col[n] = make_int4(ry * tw + rx, e.y, e.z, (e.x % W) | ((e.x / W) << 16));
                const int ax = e.y % W - d.x0, ay = e.y / W - d.y0;
                const int plane = (ax >= 0 && ax < kPW && ay >= 0 && ay < kPH) ? ay * kPW + ax : -1;
                col1[n] = make_int4(rx + kPW / 2, ry + kPH / 2, plane, 0);
            }
            if (!colpath)
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
                if (colpath) {
                    // transpose 32 columns through shared memory; warp w then sums, for the
                    // column of each lane, its quarter of the 112 stencil offsets
                    const int lane = et & 31;
#pragma unroll
                    for (int i = 0; i < 32; ++i) dt[i * kTcM + et] = __uint_as_float(v[i]);
                    epi_sync();
                    int a[kCls6];
#pragma unroll
                    for (int c = 0; c < kCls6; ++c) a[c] = 0;
                    if (c0 + lane < nn) {
                        const int4 c1 = col1[c0 + lane];
                        const float *dtc = dt + lane * kTcM;
                        stencil_warp(w, dtc, c1, lane, a);
                    }
#pragma unroll
                    for (int c = 0; c < kCls6; ++c) part[(w * 32 + lane) * 33 + c] = a[c];
                    epi_sync();
                    // sums of the four quarters: warp w takes columns w, w + 4, ...; lane = class
                    for (int cl = w; cl < 32; cl += 4) {
                        const int n = c0 + cl;
                        if (n < nn && lane < kCls6) {
                            const int sum = part[cl * 33 + lane] + part[(32 + cl) * 33 + lane] +
                                            part[(64 + cl) * 33 + lane] +
                                            part[(96 + cl) * 33 + lane];
                            const int slot = col[n].z;  // the b side carries -delta
                            if (sum)
                                red_add_global(side + (size_t)slot * kMaxClasses + lane,
                                               (slot & 1) ? -sum : sum);
                        }
                    }
                } else if (qin && fast) {
                    // per 16 columns: the table lookups first (independent loads), then the
                    // class-sum updates
#pragma unroll
                    for (int h = 0; h < 32; h += 16) {
                        int cls[16];
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const int n = c0 + h + i < nn ? c0 + h + i : nn - 1;
                            const int2 ci = *reinterpret_cast<const int2 *>(col + n);
                            const int c = tab2[lt - ci.x];
                            cls[i] = (c0 + h + i < nn && qpix != ci.y) ? c : -1;
                        }
#pragma unroll
                        for (int i = 0; i < 16; ++i)
                            if (cls[i] >= 0)
                                atomicAdd(&acc[(c0 + h + i) * 32 + cls[i]],
                                          __float2int_rn(__uint_as_float(v[h + i])));
                    }
                } else if (qin) {
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const int n = c0 + i;
                        if (n < nn) {
                            const int4 ci = col[n];
                            int dx = qx - (ci.w & 0xFFFF), dy = qy - (ci.w >> 16);
                            dx += dx < -hw ? W : 0;
                            dx -= dx > hw ? W : 0;
                            dy += dy < -hh ? H : 0;
                            dy -= dy > hh ? H : 0;
                            const int d2 = dx * dx + dy * dy;  // |dx| <= W/2, |dy| <= H/2
                            if (d2 <= r2) {
                                const int c = tab[d2];  // -1 for d2 = 0 and empty classes
                                if (c >= 0 && qpix != ci.y)
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
            // warp w sends the class sums of columns w, w + 4, ...; lane = class
            if (!colpath) {
                const int lane = et & 31;
                for (int nb = w; nb < nn; nb += 4 * kFlushBatch) {
                    int val[kFlushBatch], slot[kFlushBatch];
#pragma unroll
                    for (int k = 0; k < kFlushBatch; ++k) {
                        const int n = nb + 4 * k;
                        slot[k] = n < nn ? col[n].z : 0;
                        val[k] = (n < nn && lane < ncls) ? acc[n * 32 + lane] : 0;
                        if (slot[k] & 1) val[k] = -val[k];  // the b side carries -delta
                    }
#pragma unroll
                    for (int k = 0; k < kFlushBatch; ++k)
                        if (val[k]) red_add_global(side + (size_t)slot[k] * kMaxClasses + lane, val[k]);
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
            mbar_init(&full[i], kProdWarps);
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

// One warp per couple: the couple's class sums are cleared, its f16 delta row k_b - k_a is
// written for every stage, and each of its two pixels is appended to the lists of the patches
// within the radius of it (lanes 0-15: pixel a, 16-31: pixel b, one patch per lane).
__global__ void __launch_bounds__(kListThreads) k_tc_lists(const Problem *probs)
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
    // deltas, 16 integrands (two f16 pieces of one stage) per lane and step
    const int nv = (pb.row_bytes >> 6) * 4;
    for (int v = lane; v < nv; v += 32) {
        const int e0 = v * 16;  // first integrand
        const size_t cb = ((size_t)(e0 >> 7) * pb.P) << 7;
        const uint4 ka = *reinterpret_cast<const uint4 *>(pb.counts + cb + ((size_t)a << 7) +
                                                          (e0 & 127));
        const uint4 kb = *reinterpret_cast<const uint4 *>(pb.counts + cb + ((size_t)b << 7) +
                                                          (e0 & 127));
        uint4 o0, o1;
        bytes_sub_h2(kb.x, ka.x, o0.x, o0.y);
        bytes_sub_h2(kb.y, ka.y, o0.z, o0.w);
        bytes_sub_h2(kb.z, ka.z, o1.x, o1.y);
        bytes_sub_h2(kb.w, ka.w, o1.z, o1.w);
        uint4 *dst = reinterpret_cast<uint4 *>(pb.tc_delta16 + (((size_t)(v >> 2) * pb.M + j) << 6) +
                                               (v & 3) * 16);
        dst[0] = o0;
        dst[1] = o1;
    }
    // lanes 0..15 list pixel a, lanes 16..31 pixel b, one patch each, all atomics in parallel
    const int side = lane >> 4, k = lane & 15;
    const int r = pb.radius, r2 = r * r;
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
    // at most 3 x 4 patches for radius <= 8; the loop covers any count
    for (int kk = k; kk < nx * ny; kk += 16) {
        const int u = kk / ny, w = kk - (kk / ny) * ny;  // this lane's patch
        if (xd[u] * xd[u] + yd[w] * yd[w] <= r2) {  // in reach
            const int pid = yi[w] * pb.tc_npx + xi[u];
            const int pos = atomicAdd(pb.tc_cnt + pid, 1);
            // min-image offset of p from the patch centre
            int rx = px - (xi[u] * kPW + kPW / 2), ry = py - (yi[w] * kPH + kPH / 2);
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

// f16 copy of the counts: piece v of the copy = 8 integrands of one pixel and stage
__global__ void k_tc_refresh(const Problem *probs)
{
    const Problem &pb = *probs;
    const long long n = (long long)pb.P * (pb.row_bytes >> 6) * 8;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        const long long per = (long long)pb.P * 8;
        const int ks = (int)(v / per);
        const int rem = (int)(v - (long long)ks * per);
        const int p = rem >> 3, pc = rem & 7;
        const int e0 = ks * 64 + pc * 8;
        const uint2 k = *reinterpret_cast<const uint2 *>(
            pb.counts + ((((size_t)(e0 >> 7) * pb.P) + p) << 7) + (e0 & 127));
        uint4 o;
        bytes_to_h2(k.x, kBiasCount, o.x, o.y);
        bytes_to_h2(k.y, kBiasCount, o.z, o.w);
        *reinterpret_cast<uint4 *>(pb.tc_counts16 + (((size_t)ks * pb.P + p) << 6) + pc * 8) = o;
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

cudaError_t launch_tc_refresh(const Problem *dprob, const std::vector<Problem> &hp,
                              cudaStream_t st)
{
    for (size_t i = 0; i < hp.size(); ++i) {
        const long long n = (long long)hp[i].P * (hp[i].row_bytes >> 6) * 8;
        const long long blocks = (n + 255) / 256;
        k_tc_refresh<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(dprob + i);
    }
    note_launches((long long)hp.size());
    return cudaGetLastError();
}

cudaError_t prepare_tc()
{
    return cudaFuncSetAttribute(k_tc_stencil, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kSmemBytes);
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
        const TcArgs a{tl.dprob, tl.n_prob, tl.unit_start, tl.total_units};
        const int grid = tl.total_units < tl.sms ? tl.total_units : tl.sms;
        if (timed) tm->begin(kKTcStencil, st);
        k_tc_stencil<<<grid, kTcThreads, kSmemBytes, st>>>(a);
        if (timed) tm->end(st);
        note_launches(1);
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
