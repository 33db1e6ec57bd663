/*
 * bn_oracle.c — plain, slow, FP64 CPU oracle for the screen-space sampler optimizer of
 * Belcour & Heitz, "Lessons Learned and Improvements when Building Screen-Space Samplers
 * with Blue-Noise Error Distribution" (SIGGRAPH '21 Talks).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or calls this file.
 * It may be used by the tests, by the smoke check and by the benchmark's CPU-baseline arm.
 * It shares no code, header, table or constant generator with the CUDA path.
 *
 * Every function is written from the paper's definitions (section / equation cited in each
 * comment), in double precision where real numbers are involved.  Where the paper leaves a
 * choice open, the reading taken is stated beside the code; the design notes list them all.
 *
 * Conventions used throughout (they are the method's interface, not an optimisation):
 *   - tile W x H pixels, toroidal; pixel p = y*W + x; P = W*H; Phat = 2^L >= P.
 *   - N = 2^m lattice points; counts k_p[t] are integers in [0, N], estimate = k/N.
 *   - all random draws come from Philox4x32-10 keyed by the 64-bit seed, with the counter
 *     (index, aux, tag, pair); tags below.
 *
 * Parity status: every function below is pinned by a CPU test against closed forms,
 * invariants, the paper's printed teaser points or an independent brute force.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define TAG_SHIFT 1u    /* per-pixel Cranley-Patterson shift u_p          */
#define TAG_HEAVI 2u    /* random Heaviside test integrands               */
#define TAG_PKEY 3u     /* round keys of the candidate permutation        */
#define TAG_PBIT 4u     /* round decisions of the candidate permutation   */
#define TAG_XOR 5u      /* per-pass XOR scramble of pixel indices         */
#define TAG_PRIO 6u     /* priority of a couple among interacting couples */

/* ------------------------------------------------------------------------------------------
 * Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, "Parallel Random
 * Numbers: As Easy as 1, 2, 3", SC'11).  Ten rounds of two 32x32->64 multiplies; the key is
 * bumped by the Weyl constants between rounds.
 * ------------------------------------------------------------------------------------------ */
void bno_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c[1] ^ k0;
        uint32_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

static void draw(uint64_t seed, uint32_t index, uint32_t aux, uint32_t tag, uint32_t pair,
                 uint32_t out[4])
{
    uint32_t ctr[4] = {index, aux, tag, pair};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    bno_philox(ctr, key, out);
}

/* ------------------------------------------------------------------------------------------
 * Main sequence (Sec. 3.2): rank-1 lattice s^k = mod(Phi(k) * d, 1), Phi = van der Corput
 * radical inverse in base 2.  The direction vector d = (1, g) is a Korobov vector; the paper's
 * own vectors are not available, so g maximises the toroidal minimum distance between lattice
 * points among g coprime to N, ties going to the smallest g.
 * ------------------------------------------------------------------------------------------ */
double bno_van_der_corput(uint32_t k)
{
    double phi = 0.0, scale = 0.5;
    while (k) {
        if (k & 1u) phi += scale;
        k >>= 1;
        scale *= 0.5;
    }
    return phi;
}

static uint32_t gcd_u32(uint32_t a, uint32_t b)
{
    while (b) { uint32_t t = a % b; a = b; b = t; }
    return a;
}

/* min over lattice points k != 0 of the squared toroidal distance to the origin, in units
 * of 1/N (the lattice is a group, so this is the minimum over all pairs of points). */
int64_t bno_korobov_min_dist2(int32_t N, int32_t g)
{
    int64_t best = INT64_MAX;
    for (int32_t k = 1; k < N; ++k) {
        int64_t x = k, y = ((int64_t)k * g) % N;
        int64_t dx = x < N - x ? x : N - x;
        int64_t dy = y < N - y ? y : N - y;
        int64_t d2 = dx * dx + dy * dy;
        if (d2 < best) best = d2;
    }
    return best;
}

int32_t bno_pick_g(int32_t N)
{
    int32_t best_g = 1;
    int64_t best = -1;
    for (int32_t g = 1; g < N; ++g) {
        if (gcd_u32((uint32_t)g, (uint32_t)N) != 1u) continue;
        int64_t d = bno_korobov_min_dist2(N, g);
        if (d > best) { best = d; best_g = g; }
    }
    return best_g;
}

/* Scrambled sequence of one pixel (Sec. 2 and Sec. 3.2): s^k_p = mod(s^k + u_p, 1). */
void bno_points(int32_t N, int32_t g, double ux, double uy, double *x, double *y)
{
    for (int32_t k = 0; k < N; ++k) {
        double phi = bno_van_der_corput((uint32_t)k);
        double sx = phi - floor(phi);                       /* mod(Phi(k) * 1, 1) */
        double sy = phi * (double)g - floor(phi * (double)g); /* mod(Phi(k) * g, 1) */
        double px = sx + ux, py = sy + uy;
        x[k] = px - floor(px);
        y[k] = py - floor(py);
    }
}

/* ------------------------------------------------------------------------------------------
 * Tile of scrambling parameters U = {u_p} (Sec. 2): one uniform shift in [0,1)^2 per pixel.
 * Stored as 0.32 fixed point with the low 8 bits cleared, so that u = U * 2^-32 is exact in
 * both float and double; the shifted points then have 24 fractional bits.
 * ------------------------------------------------------------------------------------------ */
void bno_shifts(uint64_t seed, int32_t pair, int32_t P, uint32_t *U /* [P][2] */)
{
    for (int32_t p = 0; p < P; ++p) {
        uint32_t r[4];
        draw(seed, (uint32_t)p, 0u, TAG_SHIFT, (uint32_t)pair, r);
        U[2 * p + 0] = r[0] & 0xFFFFFF00u;
        U[2 * p + 1] = r[1] & 0xFFFFFF00u;
    }
}

/* ------------------------------------------------------------------------------------------
 * Test integrands (Sec. 2, Fig. 1b): randomly oriented Heavisides f(x) = [a x + b y < c].
 * Orientation: integer normal (a, b) uniform in the disc of radius 2^15 (rejection from the
 * square); offset c uniform over the range a x + b y takes on the unit square, so the edge
 * always crosses the square.  c is stored as C = c * 2^24 (an integer).
 * ------------------------------------------------------------------------------------------ */
void bno_heaviside_bank(uint64_t seed, int32_t pair, int32_t T, int32_t *a, int32_t *b,
                        int64_t *C)
{
    for (int32_t t = 0; t < T; ++t) {
        int32_t ai = 1, bi = 0;
        uint32_t roff = 0x80000000u;
        for (uint32_t attempt = 0; attempt < 64u; ++attempt) {
            uint32_t r[4];
            draw(seed, (uint32_t)t, attempt, TAG_HEAVI, (uint32_t)pair, r);
            int32_t ca = (int32_t)(r[0] >> 16) - 32768;
            int32_t cb = (int32_t)(r[1] >> 16) - 32768;
            int64_t q = (int64_t)ca * ca + (int64_t)cb * cb;
            if (q > 0 && q <= ((int64_t)1 << 30)) {
                ai = ca; bi = cb; roff = r[2];
                break;
            }
        }
        int64_t lo = (ai < 0 ? ai : 0) + (bi < 0 ? bi : 0);
        int64_t hi = (ai > 0 ? ai : 0) + (bi > 0 ? bi : 0);
        /* c = lo + (hi - lo) * roff / 2^32, scaled by 2^24 and rounded down */
        uint64_t span = (uint64_t)(hi - lo);
        a[t] = ai;
        b[t] = bi;
        C[t] = lo * ((int64_t)1 << 24) + (int64_t)(((uint64_t)roff * span) >> 8);
    }
}

/* ------------------------------------------------------------------------------------------
 * Candidate permutation (Sec. 3.4): a permutation of pixel indices stored in a linear array.
 * The paper does not say how it is drawn; here it is the swap-or-not shuffle of Hoang,
 * Morris and Rogaway (CRYPTO 2012) on the domain [0, 2^L): each round XORs with a round key
 * K_r and swaps x with x ^ K_r when a random bit attached to the pair {x, x ^ K_r} is set.
 * ------------------------------------------------------------------------------------------ */
int32_t bno_perm_rounds(int32_t L)
{
    int32_t r = 6 * L;
    return r < 12 ? 12 : r;
}

void bno_permutation(uint64_t seed, int32_t pair, int32_t L, int32_t *perm /* [2^L] */)
{
    uint32_t n = 1u << L, mask = n - 1u;
    int32_t rounds = bno_perm_rounds(L);
    for (uint32_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    for (int32_t r = 0; r < rounds; ++r) {
        uint32_t kr[4];
        draw(seed, (uint32_t)r, 0u, TAG_PKEY, (uint32_t)pair, kr);
        uint32_t K = kr[0] & mask;
        for (uint32_t i = 0; i < n; ++i) {
            uint32_t x = (uint32_t)perm[i];
            uint32_t partner = x ^ K;
            uint32_t hi = x > partner ? x : partner;
            uint32_t bit[4];
            draw(seed, hi, (uint32_t)r, TAG_PBIT, (uint32_t)pair, bit);
            if (bit[0] & 1u) perm[i] = (int32_t)partner;
        }
    }
}

/* ------------------------------------------------------------------------------------------
 * Test-integrand map (Sec. 2): k_p[t] = sum_k f_t(s^k_p), so that I_p[t] = k_p[t] / N.
 * Evaluated in double: every product and sum involved is exact (<= 41 significant bits).
 * ------------------------------------------------------------------------------------------ */
void bno_counts(int32_t N, int32_t g, int32_t P, const uint32_t *U, int32_t T,
                const int32_t *a, const int32_t *b, const int64_t *C, int32_t *k /* [P][T] */)
{
    double *x = (double *)malloc(sizeof(double) * (size_t)N);
    double *y = (double *)malloc(sizeof(double) * (size_t)N);
    const double two32 = 4294967296.0, two24 = 16777216.0;
    for (int32_t p = 0; p < P; ++p) {
        bno_points(N, g, (double)U[2 * p] / two32, (double)U[2 * p + 1] / two32, x, y);
        for (int32_t t = 0; t < T; ++t) {
            double c = (double)C[t] / two24;
            int32_t cnt = 0;
            for (int32_t j = 0; j < N; ++j)
                if ((double)a[t] * x[j] + (double)b[t] * y[j] < c) ++cnt;
            k[(size_t)p * T + t] = cnt;
        }
    }
    free(x);
    free(y);
}

/* ------------------------------------------------------------------------------------------
 * Neighbourhood on the torus.  Eq. 1 sums over all q != p; the weight is truncated at
 * distance r and distances are min-image distances on the toroidal tile.  Each distinct
 * pixel q is visited once, even on tiles smaller than 2r+1.
 * canonical(d, W): d is the min-image representative of its residue (ties -> +W/2).
 * ------------------------------------------------------------------------------------------ */
static int canonical(int32_t d, int32_t W)
{
    int32_t o = ((d % W) + W) % W;
    int32_t rep = (2 * o <= W) ? o : o - W;
    return rep == d;
}

static int32_t wrap(int32_t v, int32_t n) { return ((v % n) + n) % n; }

/* min-image squared distance between pixels p and q */
int32_t bno_torus_d2(int32_t W, int32_t H, int32_t p, int32_t q)
{
    int32_t ox = wrap(q % W - p % W, W), oy = wrap(q / W - p / W, H);
    int32_t dx = ox < W - ox ? ox : W - ox;
    int32_t dy = oy < H - oy ? oy : H - oy;
    return dx * dx + dy * dy;
}

/* weight of Eq. 1: exp(-d^2 / sigma^2) (sigma = 2.1 in the paper, used literally) */
static double weight(int32_t d2, double sigma) { return exp(-(double)d2 / (sigma * sigma)); }

/* ------------------------------------------------------------------------------------------
 * Loss, Eq. 1: L = sum_p sum_{q != p} exp(-|p-q|^2 / sigma^2) |I_p - I_q|^2, over ordered
 * pairs within distance r, I = k / N.  Direct double loop over p and its distinct neighbours.
 * Optionally returns the exact integer sum of |k_p - k_q|^2 per squared distance d2.
 * ------------------------------------------------------------------------------------------ */
double bno_energy(int32_t W, int32_t H, int32_t N, int32_t T, const int32_t *k, double sigma,
                  int32_t r, int64_t *class_sum /* [r*r+1] or NULL */)
{
    double E = 0.0;
    if (class_sum) memset(class_sum, 0, sizeof(int64_t) * (size_t)(r * r + 1));
    for (int32_t py = 0; py < H; ++py)
        for (int32_t px = 0; px < W; ++px) {
            const int32_t *kp = k + ((size_t)py * W + px) * T;
            for (int32_t dy = -r; dy <= r; ++dy)
                for (int32_t dx = -r; dx <= r; ++dx) {
                    if (dx == 0 && dy == 0) continue;
                    if (dx * dx + dy * dy > r * r) continue;
                    if (!canonical(dx, W) || !canonical(dy, H)) continue;
                    const int32_t *kq = k + ((size_t)wrap(py + dy, H) * W + wrap(px + dx, W)) * T;
                    int64_t s = 0;
                    for (int32_t t = 0; t < T; ++t) {
                        int64_t d = (int64_t)kp[t] - kq[t];
                        s += d * d;
                    }
                    int32_t d2 = dx * dx + dy * dy;
                    if (class_sum) class_sum[d2] += s;
                    E += weight(d2, sigma) * (double)s / ((double)N * (double)N);
                }
        }
    return E;
}

/* ------------------------------------------------------------------------------------------
 * Energy change of one move (Sec. 2 and Sec. 3.4): the move swaps the scrambling values of
 * pixels a and b, which swaps their estimate vectors.  Only the terms of Eq. 1 that involve a
 * or b change; they are summed before and after the swap, per squared distance d2.
 * dE_class[d2] receives the change of those terms of distance d2; the return value is their
 * sum.  Both orders of each pair are counted, as in Eq. 1.
 * ------------------------------------------------------------------------------------------ */
static int64_t sqdist(const int32_t *u, const int32_t *v, int32_t T)
{
    int64_t s = 0;
    for (int32_t t = 0; t < T; ++t) {
        int64_t d = (int64_t)u[t] - v[t];
        s += d * d;
    }
    return s;
}

/* integer sums, per d2, of |k_p - k_q|^2 over ordered pairs that involve a or b, with the
 * estimate vectors of a and b given explicitly (ka at pixel a, kb at pixel b) */
static void local_terms(int32_t W, int32_t H, int32_t T, const int32_t *k, int32_t r,
                        int32_t a, int32_t b, const int32_t *ka, const int32_t *kb,
                        int64_t *acc /* [r*r+1] */)
{
    const int32_t centre[2] = {a, b};
    for (int32_t side = 0; side < 2; ++side) {
        int32_t p = centre[side];
        const int32_t *kp = side == 0 ? ka : kb;
        int32_t px = p % W, py = p / W;
        for (int32_t dy = -r; dy <= r; ++dy)
            for (int32_t dx = -r; dx <= r; ++dx) {
                if (dx == 0 && dy == 0) continue;
                if (dx * dx + dy * dy > r * r) continue;
                if (!canonical(dx, W) || !canonical(dy, H)) continue;
                int32_t q = wrap(py + dy, H) * W + wrap(px + dx, W);
                const int32_t *kq = k + (size_t)q * T;
                if (q == a) kq = ka;
                if (q == b) kq = kb;
                int64_t s = sqdist(kp, kq, T);
                /* the pair (p, q) and the pair (q, p) */
                if (side == 1 && q == a) continue; /* {a, b} already counted from a's side */
                acc[dx * dx + dy * dy] += 2 * s;
            }
    }
}

double bno_delta_energy(int32_t W, int32_t H, int32_t N, int32_t T, const int32_t *k,
                        double sigma, int32_t r, int32_t a, int32_t b,
                        double *dE_class /* [r*r+1] or NULL */)
{
    int32_t nc = r * r + 1;
    int64_t *before = (int64_t *)calloc((size_t)nc, sizeof(int64_t));
    int64_t *after = (int64_t *)calloc((size_t)nc, sizeof(int64_t));
    const int32_t *ka = k + (size_t)a * T, *kb = k + (size_t)b * T;
    local_terms(W, H, T, k, r, a, b, ka, kb, before);
    local_terms(W, H, T, k, r, a, b, kb, ka, after); /* swapped */
    double dE = 0.0;
    for (int32_t c = 0; c < nc; ++c) {
        double v = weight(c, sigma) * (double)(after[c] - before[c]) / ((double)N * (double)N);
        if (dE_class) dE_class[c] = v;
        dE += v;
    }
    free(before);
    free(after);
    return dE;
}

/* ------------------------------------------------------------------------------------------
 * One optimisation pass (Sec. 3.4).
 *   1. Candidates: the precomputed permutation, with every stored pixel index XORed by a
 *      per-pass value x_s; couple j = (perm[2j] ^ x_s, perm[2j+1] ^ x_s), j < M.  A couple with
 *      an index outside the tile (padding of P up to 2^L) is dropped.
 *   2. Each couple's energy change is evaluated on the unmodified tile.
 *   3. Acceptance as in the sequential optimiser: a swap is kept only if it improves the
 *      objective.  objective = +1 reduces Eq. 1 as printed; objective = -1 raises Eq. 1.  A swap
 *      keeps sum_p |I_p|^2 fixed, so raising Eq. 1 is the same as lowering the Gaussian-weighted
 *      correlation sum_p sum_q w I_p.I_q of neighbouring estimates, which is what spreads the
 *      error as blue noise (the criterion of Sec. 3.3 improves; reducing Eq. 1 literally makes
 *      neighbouring estimates alike and the criterion worsens).  -1 is the default reading.
 *   4. Couples never share a pixel.  In addition, among improving couples that interact (a
 *      pixel of one within distance r of a pixel of the other), only the one of highest
 *      priority (Philox draw, then lower j) is kept, so the kept changes add up exactly.
 *   5. The kept swaps are applied to the estimate vectors and the shift index of the tile.
 * dE[j] is the change of Eq. 1 (not of the objective); improving means objective * dE < 0.
 * mode = 1 (concurrent) keeps every improving couple, with no interaction filter: this is the
 * paper's own GPU optimiser, whose loss can move the wrong way while many neighbouring swaps
 * land in the same pass.
 * Lockstep use: if gpu_improving is given, couples whose |dE| is below tie_rel * S_j (S_j = sum
 * of the absolute per-distance changes) take their improving flag from it instead; such
 * couples are flagged in flags bit 3.
 * flags bits: 1 = valid, 2 = improving, 4 = committed, 8 = tie.
 * ------------------------------------------------------------------------------------------ */
static int interact(int32_t W, int32_t H, int32_t r, int32_t a0, int32_t b0, int32_t a1,
                    int32_t b1)
{
    int32_t r2 = r * r;
    return bno_torus_d2(W, H, a0, a1) <= r2 || bno_torus_d2(W, H, a0, b1) <= r2 ||
           bno_torus_d2(W, H, b0, a1) <= r2 || bno_torus_d2(W, H, b0, b1) <= r2;
}

void bno_sweep_couples(uint64_t seed, int32_t pair, uint32_t sweep, int32_t L, int32_t M,
                       const int32_t *perm, int32_t *couples /* [M][2] */)
{
    uint32_t r[4];
    draw(seed, sweep, 0u, TAG_XOR, (uint32_t)pair, r);
    uint32_t xs = r[0] & ((1u << L) - 1u);
    for (int32_t j = 0; j < M; ++j) {
        couples[2 * j] = (int32_t)((uint32_t)perm[2 * j] ^ xs);
        couples[2 * j + 1] = (int32_t)((uint32_t)perm[2 * j + 1] ^ xs);
    }
}

uint64_t bno_priority_key(uint64_t seed, int32_t pair, uint32_t sweep, int32_t j)
{
    uint32_t r[4];
    draw(seed, (uint32_t)j, sweep, TAG_PRIO, (uint32_t)pair, r);
    return ((uint64_t)r[0] << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)j);
}

int32_t bno_sweep(int32_t W, int32_t H, int32_t N, int32_t T, double sigma, int32_t r,
                  int32_t objective, int32_t mode, uint64_t seed, int32_t pair, uint32_t sweep, int32_t L,
                  int32_t M, const int32_t *perm, int32_t *k /* [P][T] in/out */,
                  int32_t *sidx /* [P] in/out */, const uint8_t *gpu_improving /* [M] or NULL */,
                  double tie_rel, double *dE /* [M] */, double *S /* [M] */,
                  uint8_t *flags /* [M] */, int32_t *couples /* [M][2] */)
{
    int32_t P = W * H, nc = r * r + 1;
    double *cls = (double *)malloc(sizeof(double) * (size_t)nc);
    bno_sweep_couples(seed, pair, sweep, L, M, perm, couples);
    for (int32_t j = 0; j < M; ++j) {
        int32_t a = couples[2 * j], b = couples[2 * j + 1];
        flags[j] = 0;
        dE[j] = 0.0;
        S[j] = 0.0;
        if (a >= P || b >= P) continue;
        flags[j] = 1;
        dE[j] = bno_delta_energy(W, H, N, T, k, sigma, r, a, b, cls);
        double s = 0.0;
        for (int32_t c = 0; c < nc; ++c) s += fabs(cls[c]);
        S[j] = s;
        int improving = (double)objective * dE[j] < 0.0;
        if (gpu_improving && fabs(dE[j]) < tie_rel * s) {
            flags[j] |= 8;
            improving = gpu_improving[j] != 0;
        }
        if (improving) flags[j] |= 2;
    }
    int32_t committed = 0;
    for (int32_t j = 0; j < M; ++j) {
        if (!(flags[j] & 2)) continue;
        if (mode == 1) {
            flags[j] |= 4;
            continue;
        }
        uint64_t kj = bno_priority_key(seed, pair, sweep, j);
        int wins = 1;
        for (int32_t i = 0; i < M && wins; ++i) {
            if (i == j || !(flags[i] & 2)) continue;
            if (!interact(W, H, r, couples[2 * i], couples[2 * i + 1], couples[2 * j],
                          couples[2 * j + 1]))
                continue;
            if (bno_priority_key(seed, pair, sweep, i) > kj) wins = 0;
        }
        if (wins) flags[j] |= 4;
    }
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (size_t)T);
    for (int32_t j = 0; j < M; ++j) {
        if (!(flags[j] & 4)) continue;
        int32_t a = couples[2 * j], b = couples[2 * j + 1];
        memcpy(tmp, k + (size_t)a * T, sizeof(int32_t) * (size_t)T);
        memcpy(k + (size_t)a * T, k + (size_t)b * T, sizeof(int32_t) * (size_t)T);
        memcpy(k + (size_t)b * T, tmp, sizeof(int32_t) * (size_t)T);
        int32_t s = sidx[a];
        sidx[a] = sidx[b];
        sidx[b] = s;
        ++committed;
    }
    free(tmp);
    free(cls);
    return committed;
}
