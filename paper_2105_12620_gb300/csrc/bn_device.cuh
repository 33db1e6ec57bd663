// bn_device.cuh — device-side data layout and helpers shared by the sampler's CUDA kernels.
//
// Layout of one problem (one 2-D pair of one tile) in device memory:
//   counts   chunk-major planes [row_bytes / 128][P][128 B]: bytes [128 c, 128 c + 128) of pixel
//            p's count vector k_p (uint8 or uint16 per integrand, zero-padded to 128 B) live at
//            counts + (c * P + p) * 128, so one chunk of a run of pixels of an image row is
//            contiguous
//   U        uint32 [P][2]    initial shifts u_p in 0.32 fixed point (low 8 bits zero)
//   sidx     int32  [P]       index of the initial shift now at pixel p (a swap moves it)
//   perm     int32  [2^L]     candidate permutation (Sec. 3.4), perm_inv its inverse
//   ha, hb   int32  [T], hC int64 [T]  Heaviside [a x + b y < c], C = c * 2^24
//   owner    uint64 [2][P]    per-pass claim of a pixel by an improving couple (by parity)
//   tc_cnt, tc_list           per-pass lists of the proposed pixels near each 16 x 8 patch
//   log_*    [M]              last pass: change of Eq. 1, flags, couple pixels
//   ctr      int64 [4]        pass counter, pass end, launch ticket, spare
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace bn {

constexpr int kMaxClasses = 32;    // radius <= 8: at most 29 distinct squared distances
constexpr int kMaxOffsets = 200;   // radius 8: 196 neighbours
constexpr int kMaxRowBytes = 4096; // T * count_bytes, padded
constexpr int kRowAlign = 128;

constexpr uint32_t kTagShift = 1u, kTagHeavi = 2u, kTagPermKey = 3u, kTagPermBit = 4u,
                   kTagXor = 5u, kTagPrio = 6u;

constexpr uint8_t kFlagValid = 1, kFlagImproving = 2, kFlagCommitted = 4, kFlagTie = 8;

enum StatIndex { kStatValid = 0, kStatImproving = 1, kStatCommitted = 2, kStatTies = 3,
                 kStatSweeps = 4, kStatError = 5, kStatCount = 8 };

struct Problem {
    int32_t W, H, P, L;
    int32_t M;                 // couples per pass
    int32_t N, m, g;           // N = 2^m points, Korobov generator g
    int32_t T, row_bytes, count_bytes;
    int32_t radius, n_off, n_cls;
    int32_t mode, objective;
    uint32_t pair;
    uint32_t seed_lo, seed_hi;
    float scale;               // 4 / N^2 (a power of two)
    float w[kMaxClasses];      // fp32 weight exp(-d2 / sigma^2) of each class
    int32_t d2[kMaxClasses];   // squared distance of each class
    int32_t cls_start[kMaxClasses + 1];  // offsets are sorted by class
    int32_t off[kMaxOffsets];  // (dx & 0xFFFF) | (dy << 16), signed min-image offsets

    uint8_t *counts;
    uint32_t *U;
    int32_t *sidx;
    int32_t *perm, *perm_inv;
    int32_t *ha, *hb;
    int64_t *hC;
    unsigned long long *owner;
    float *log_dE;
    uint8_t *log_flags;
    int32_t *log_couples;
    int32_t *side_cls;         // [M][2 x tsplit][kMaxClasses] partial class sums (persistent);
                               // [2 M][kMaxClasses] per proposed pixel (tensor-core schedule)
    int32_t *tc_cnt;           // [tc_npx * tc_npy] proposed pixels listed per patch
    int4 *tc_list;             // [tc_npx * tc_npy][tc_cap] (pixel, partner, slot 2 j + side,
                               // position relative to the patch centre), see bn_tc.cu
    int32_t tc_npx, tc_npy, tc_cap;  // patches of 16 x 8 pixels per row / column, list capacity
    // tensor-core schedule only (owned by its plan, null elsewhere): per-pass f16 deltas
    // k_b - k_a of the couples, [stages][M][64] with stages = row_bytes / (64 count_bytes)
    uint16_t *tc_delta16;
    long long *ctr;            // [0] pass counter, [1] pass end, [2] ticket
    unsigned long long *stats; // [kStatCount]
    unsigned long long *esum;  // [kMaxClasses] energy class sums (two's complement int64)
    double *energy_out;
};

// ---------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): counter (index, aux, tag, pair), key = 64-bit seed.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return make_uint4(c0, c1, c2, c3);
}

__device__ __forceinline__ uint4 draw(const Problem &pb, uint32_t index, uint32_t aux,
                                      uint32_t tag)
{
    return philox(index, aux, tag, pb.pair, pb.seed_lo, pb.seed_hi);
}

// per-pass XOR value applied to every stored candidate index (Sec. 3.4)
__device__ __forceinline__ uint32_t pass_xor(const Problem &pb, uint32_t sweep)
{
    return draw(pb, sweep, 0u, kTagXor).x & ((1u << pb.L) - 1u);
}

// priority among interacting improving couples: (Philox draw, then lower index wins)
__device__ __forceinline__ unsigned long long couple_key(const Problem &pb, uint32_t sweep,
                                                         int32_t j)
{
    const uint32_t r = draw(pb, (uint32_t)j, sweep, kTagPrio).x;
    return ((unsigned long long)r << 32) | (unsigned long long)(0xFFFFFFFFu - (uint32_t)j);
}

__device__ __forceinline__ int wrap_add(int v, int d, int n)
{
    v += d;
    v += (v < 0) ? n : 0;
    v -= (v >= n) ? n : 0;
    return v;
}

// chunk c of pixel p's count vector (128 bytes)
__device__ __forceinline__ uint8_t *chunk_ptr(const Problem &pb, int p, int c)
{
    return pb.counts + (((size_t)c * pb.P + p) << 7);
}

// 16-byte piece vi (0 <= vi < row_bytes / 16) of pixel p's count vector
__device__ __forceinline__ uint4 *vec_ptr(const Problem &pb, int p, int vi)
{
    return reinterpret_cast<uint4 *>(pb.counts + (((size_t)(vi >> 3) * pb.P + p) << 7) +
                                     ((vi & 7) << 4));
}

// neighbour of pixel p at table offset i
__device__ __forceinline__ int neighbour(const Problem &pb, int px, int py, int i)
{
    const int o = pb.off[i];
    const int dx = (int)(int16_t)(o & 0xFFFF), dy = o >> 16;
    return wrap_add(py, dy, pb.H) * pb.W + wrap_add(px, dx, pb.W);
}

// ---------------------------------------------------------------------------------------------
// Integer dot products of packed count words.
//   8-bit rows: 4 counts per word; delta words hold signed byte differences (|d| <= 64).
//   16-bit rows: 2 counts per word; delta words hold signed 16-bit differences.
// ---------------------------------------------------------------------------------------------
template <int CB>
__device__ __forceinline__ int dot_word(uint32_t d, uint32_t k, int acc);

template <>
__device__ __forceinline__ int dot_word<1>(uint32_t d, uint32_t k, int acc)
{
    return __dp4a((int)d, (int)k, acc);
}

template <>
__device__ __forceinline__ int dot_word<2>(uint32_t d, uint32_t k, int acc)
{
    acc += (int)(int16_t)(d & 0xFFFFu) * (int)(k & 0xFFFFu);
    acc += ((int)d >> 16) * (int)(k >> 16);
    return acc;
}

template <int CB>
__device__ __forceinline__ int dot_vec(uint4 d, uint4 k, int acc)
{
    acc = dot_word<CB>(d.x, k.x, acc);
    acc = dot_word<CB>(d.y, k.y, acc);
    acc = dot_word<CB>(d.z, k.z, acc);
    acc = dot_word<CB>(d.w, k.w, acc);
    return acc;
}

// per-lane difference of packed counts: partner - self
template <int CB>
__device__ __forceinline__ uint32_t sub_word(uint32_t partner, uint32_t self);
template <>
__device__ __forceinline__ uint32_t sub_word<1>(uint32_t partner, uint32_t self)
{
    return __vsub4(partner, self);
}
template <>
__device__ __forceinline__ uint32_t sub_word<2>(uint32_t partner, uint32_t self)
{
    return __vsub2(partner, self);
}
template <int CB>
__device__ __forceinline__ uint4 sub_vec(uint4 partner, uint4 self)
{
    return make_uint4(sub_word<CB>(partner.x, self.x), sub_word<CB>(partner.y, self.y),
                      sub_word<CB>(partner.z, self.z), sub_word<CB>(partner.w, self.w));
}

// sum of squared differences of packed counts
template <int CB>
__device__ __forceinline__ int sqdiff_word(uint32_t a, uint32_t b, int acc);
template <>
__device__ __forceinline__ int sqdiff_word<1>(uint32_t a, uint32_t b, int acc)
{
    const uint32_t d = __vabsdiffu4(a, b);
    return (int)__dp4a(d, d, (unsigned)acc);
}
template <>
__device__ __forceinline__ int sqdiff_word<2>(uint32_t a, uint32_t b, int acc)
{
    const uint32_t d = __vabsdiffu2(a, b);
    const int lo = (int)(d & 0xFFFFu), hi = (int)(d >> 16);
    return acc + lo * lo + hi * hi;
}

// ---------------------------------------------------------------------------------------------
// fp32 weighted sum of exact integers, sum_c w_c * A_c, with error-free transformations:
// every integer is split into float-exact parts, each product is made exact with an FMA
// (TwoProduct) and accumulated with TwoSum, so the result hi + lo is the correctly rounded
// double-float of sum_c fl32(w_c) * A_c up to O(n u^2).
// ---------------------------------------------------------------------------------------------
struct F2 {
    float hi, lo;
};

__device__ __forceinline__ void two_sum_acc(F2 &s, float x)
{
    const float t = s.hi + x;
    const float bp = t - s.hi;
    const float err = (s.hi - (t - bp)) + (x - bp);
    s.hi = t;
    s.lo += err;
}

__device__ __forceinline__ void add_product(F2 &s, float w, float x)
{
    const float p = w * x;
    const float e = __fmaf_rn(w, x, -p);
    two_sum_acc(s, p);
    s.lo += e;
}

// A: int32 (|A| < 2^31); split as A = hi * 2^12 + lo with both parts float-exact
__device__ __forceinline__ void add_weighted_i32(F2 &s, float w, int A)
{
    const int hi = A >> 12, lo = A & 0xFFF;
    add_product(s, w, (float)hi * 4096.0f);
    add_product(s, w, (float)lo);
}

// A: int64 (|A| < 2^62); three 24-bit limbs, each float-exact
__device__ __forceinline__ void add_weighted_i64(F2 &s, float w, long long A)
{
    const long long l2 = A >> 48;
    const long long l1 = (A >> 24) & 0xFFFFFF;
    const long long l0 = A & 0xFFFFFF;
    add_product(s, w, (float)l2 * 281474976710656.0f);  // 2^48
    add_product(s, w, (float)l1 * 16777216.0f);         // 2^24
    add_product(s, w, (float)l0);
}

__device__ __forceinline__ void renorm(F2 &s)
{
    const float t = s.hi + s.lo;
    s.lo = s.lo - (t - s.hi);
    s.hi = t;
}


// fp32 change of Eq. 1 from the exact class sums; also the sum of absolute terms
__device__ __forceinline__ void couple_delta(const Problem &pb, const int *A, float &dL,
                                             float &S)
{
    F2 acc = {0.f, 0.f};
    float sabs = 0.f;
#pragma unroll
    for (int c = 0; c < kMaxClasses; ++c) {
        if (c < pb.n_cls) {
            add_weighted_i32(acc, pb.w[c], A[c]);
            sabs += pb.w[c] * fabsf((float)A[c]);
        }
    }
    renorm(acc);
    dL = -pb.scale * acc.hi;
    S = pb.scale * sabs;
}

}  // namespace bn
