/*
 * bn_sample.cuh — device-side lookup of an optimised screen-space sampler, for a renderer's own
 * CUDA kernels (header only).
 *
 * Sec. 3.2: the sampler of pixel p is the rank-1 lattice s^k = mod(Phi(k) (1, g), 1), N = 2^m
 * points, shifted on the torus by the pixel's optimised u_p: s_p^k = mod(s^k + u_p, 1).
 * Sec. 3.1: blue noise holds only within a pair of dimensions, so a renderer takes dimensions in
 * pairs: dimension d reads coordinate d % 2 of the tile optimised for pair d / 2, and an effect
 * that needs a single dimension still takes a pair and ignores its second coordinate.  The tile
 * repeats over the screen: screen pixel (x, y) uses tile pixel (x mod width, y mod height).
 *
 * The shift tables come from bn_export_shift_table (one per pair, device memory, 0.32 fixed point
 * with the low 8 bits zero), so every sample is a multiple of 2^-24 and exact in float.
 */
#ifndef BN_SAMPLE_CUH
#define BN_SAMPLE_CUH

#include <stdint.h>

typedef struct bn_sample_table {
    const uint32_t *shifts[2]; /* per pair: device uint32 [height][width][2]                    */
    int32_t width, height;     /* tile size                                                      */
    int32_t n_pairs;           /* pairs of dimensions available (1 or 2)                         */
    int32_t log2_points;       /* m: N = 2^m lattice points per pixel                            */
    int32_t generator_g;       /* Korobov generator of the lattice                               */
} bn_sample_table;

/* Sample k (taken mod N) of screen pixel (x, y) in dimension dim (0 <= dim < 2 n_pairs). */
static __device__ __forceinline__ float bn_sample(const bn_sample_table &tb, int x, int y, int k,
                                                  int dim)
{
    const int px = ((x % tb.width) + tb.width) % tb.width;
    const int py = ((y % tb.height) + tb.height) % tb.height;
    const int m = tb.log2_points;
    const uint32_t kk = (uint32_t)k & ((1u << m) - 1u);
    const uint32_t rk = __brev(kk) >> (32 - m);                 /* Phi(k) 2^m */
    const uint32_t s = (dim & 1) ? ((rk * (uint32_t)tb.generator_g) & ((1u << m) - 1u)) : rk;
    const uint32_t *u = tb.shifts[dim >> 1] + 2 * ((size_t)py * tb.width + px);
    const uint32_t v = (s << (32 - m)) + u[dim & 1];           /* mod 1 in 0.32 fixed point */
    return (float)v * 2.3283064365386963e-10f;                 /* v * 2^-32, exact */
}

#endif /* BN_SAMPLE_CUH */
