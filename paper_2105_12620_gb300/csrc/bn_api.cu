// bn_api.cu — host runtime behind the C ABI declared in include/bn_sampler.h: validation,
// device memory, problem descriptors, and the call sequences of init / sweeps / fetches.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <map>
#include <mutex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "bn_launch.h"
#include "bn_persistent.h"
#include "bn_trace.h"
#include "bn_sampler.h"

namespace {

thread_local std::string g_error;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_error = buf;
    return code;
}

}  // namespace

void bn::set_last_error(const char *msg) { g_error = msg; }

namespace {

#define BN_CUDA(call)                                                                        \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail(e_ == cudaErrorMemoryAllocation ? BN_ERR_OOM : BN_ERR_CUDA,          \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,    \
                        __LINE__);                                                           \
    } while (0)

int log2_ceil(long long n)
{
    int L = 0;
    while ((1ll << L) < n) ++L;
    return L;
}

int64_t gcd64(int64_t a, int64_t b)
{
    while (b) {
        int64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// Korobov generator with the largest toroidal minimum distance (ties: smallest g), Sec. 3.2
int korobov_g(int N)
{
    int best_g = 1;
    long long best = -1;
    for (int g = 1; g < N; ++g) {
        if (gcd64(g, N) != 1) continue;
        long long d = -1;
        for (long long k = 1; k < N; ++k) {
            long long x = k, y = (k * g) % N;
            long long dx = x < N - x ? x : N - x, dy = y < N - y ? y : N - y;
            long long d2 = dx * dx + dy * dy;
            if (d < 0 || d2 < d) d = d2;
        }
        if (d > best) {
            best = d;
            best_g = g;
        }
    }
    return best_g;
}

struct Slab {
    char *base = nullptr;
    size_t used = 0, cap = 0;
    template <typename T>
    T *take(size_t n)
    {
        size_t off = (used + 255) & ~size_t(255);
        used = off + n * sizeof(T);
        return base ? reinterpret_cast<T *>(base + off) : nullptr;
    }
};

}  // namespace

namespace {

// How the passes of a set of problems are executed, and the device arrays that go with it.
struct SweepPlan {
    bool ready = false;             // built completely; a failed build leaves an empty plan
    bool persistent = false;
    bool tensor = false;            // tensor-core schedule (every problem supports it)
    int4 *d_tc_units = nullptr;     // [tc_units] (problem, patch, x0, y0) of every 16 x 8 patch
    int tc_units = 0;
    bool tc_rounds = false;         // some problem needs several accumulator rounds
    // the problems as the tensor-core kernels see them: the same state plus the plan's per-pass
    // f16 delta rows (allocations in tc_bufs)
    bn::Problem *d_tcprob = nullptr;
    std::vector<bn::Problem> tcprob;
    std::vector<void *> tc_bufs;
    bn::PersistentShape shape{8, 8, 256, 4, 0};
    // per count width (index cb - 1): first problem, problem count, units / couples prefix
    int first[2] = {0, 0}, count[2] = {0, 0};
    int total_units[2] = {0, 0}, total_couples[2] = {0, 0};
    int *d_prefix = nullptr;        // [2][2][n_prob + 1] unit / couple prefix sums
    bn::GridBarrier *d_bar = nullptr;
    int *d_work = nullptr;          // [2] phase-1 unit counters
    char *d_tmaps = nullptr;        // TMA tensor maps of the count planes (tensor-core plans)
    int n_prob = 0, max_M = 0, sms = 0;
    // plain schedule: passes per captured CUDA graph (0 = launch every kernel directly); the
    // graphs hold the problem pointers, so they live and die with the plan
    int graph_passes = 32;
    cudaStream_t capture = nullptr;     // captures cannot run on the legacy default stream
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
};

void free_graphs(SweepPlan &pl)
{
    for (auto &g : pl.graph)
        if (g) cudaGraphExecDestroy(g);
    pl.graph[0] = pl.graph[1] = nullptr;
}

void free_plan(SweepPlan &pl)
{
    if (pl.d_prefix) cudaFree(pl.d_prefix);
    if (pl.d_bar) cudaFree(pl.d_bar);
    if (pl.d_work) cudaFree(pl.d_work);
    if (pl.d_tmaps) cudaFree(pl.d_tmaps);
    if (pl.d_tc_units) cudaFree(pl.d_tc_units);
    pl.d_tc_units = nullptr;
    if (pl.d_tcprob) cudaFree(pl.d_tcprob);
    pl.d_tcprob = nullptr;
    for (void *b : pl.tc_bufs) cudaFree(b);
    pl.tc_bufs.clear();
    pl.tcprob.clear();
    pl.ready = false;
    pl.tensor = false;
    pl.persistent = false;
    pl.tc_units = 0;
    pl.tc_rounds = false;
    pl.d_prefix = nullptr;
    pl.d_bar = nullptr;
    pl.d_work = nullptr;
    pl.d_tmaps = nullptr;
    free_graphs(pl);
    if (pl.capture) cudaStreamDestroy(pl.capture);
    pl.capture = nullptr;
}

}  // namespace

struct bn_sampler {
    bn_config cfg{};
    cudaStream_t stream = nullptr;
    int device = 0;
    int n_prob = 0;
    std::vector<bn::Problem> hprob;
    bn::Problem *dprob = nullptr;
    char *slab = nullptr;
    size_t slab_bytes = 0;
    double *h_energy = nullptr;  // pinned, [n_prob]
    float *d_shifts = nullptr;   // device staging of fetched shifts [n_prob][P][2]
    float *h_shifts = nullptr;   // pinned staging of fetched shifts
    int64_t sweep = 0;           // host mirror of the pass counter
    int schedule = BN_SCHEDULE_PLAIN;
    bn::Problem *h_pinned = nullptr;  // pinned staging of the descriptors (reset)
    bn::KernelTimer timer;
    SweepPlan plan;
};

struct bn_batch {
    std::vector<bn_sampler *> members;
    std::vector<int> member_of;        // member index of each problem (grouped order)
    int *h_ends = nullptr;             // pinned, [n_prob] pass budgets
    int *d_ends = nullptr;             // device copy
    cudaStream_t stream = nullptr;
    bn::Problem *dprob = nullptr;
    int n_prob = 0;
    int max_M = 0;
    int count_bytes = 1;
    bn::KernelTimer *timer = nullptr;  // the first member's timer
    cudaEvent_t done = nullptr;        // end of the last sweep call, awaited by member streams
    std::vector<bn::Problem> all;      // host copies, grouped by count width
    SweepPlan plan;
};

namespace {

int validate(const bn_config &c)
{
    if (c.width < 2 || c.height < 2 || c.width > 4096 || c.height > 4096)
        return fail(BN_ERR_INVALID_ARG, "width/height must be in [2, 4096] (got %d x %d)",
                    c.width, c.height);
    if ((long long)c.width * c.height > (1ll << 22))
        return fail(BN_ERR_INVALID_ARG, "width*height must be <= 2^22");
    if (c.n_points < 2 || c.n_points > 1024 || (c.n_points & (c.n_points - 1)))
        return fail(BN_ERR_INVALID_ARG, "n_points must be a power of two in [2, 1024] (got %d)",
                    c.n_points);
    if (c.generator_g != 0 &&
        (c.generator_g < 1 || c.generator_g >= c.n_points || gcd64(c.generator_g, c.n_points) != 1))
        return fail(BN_ERR_INVALID_ARG, "generator_g must be 0 or coprime to N in [1, N)");
    if (c.n_pairs != 1 && c.n_pairs != 2)
        return fail(BN_ERR_INVALID_ARG, "n_pairs must be 1 or 2");
    const int cb = c.n_points <= 64 ? 1 : 2;
    if (c.n_integrands < 1 || (long long)c.n_integrands * cb > bn::kMaxRowBytes)
        return fail(BN_ERR_INVALID_ARG, "n_integrands must be in [1, %d] for N = %d",
                    bn::kMaxRowBytes / cb, c.n_points);
    if (24.0 * c.n_integrands * (double)c.n_points * c.n_points >= 2147483648.0)
        return fail(BN_ERR_INVALID_ARG, "24 * T * N^2 must be < 2^31 (exact int32 sums)");
    if (!(c.sigma > 0.f) || !std::isfinite(c.sigma))
        return fail(BN_ERR_INVALID_ARG, "sigma must be positive");
    if (c.radius < 1 || c.radius > 8) return fail(BN_ERR_INVALID_ARG, "radius must be in [1, 8]");
    const int L = log2_ceil((long long)c.width * c.height);
    if (c.couples_per_sweep < 0 || c.couples_per_sweep > (1 << L) / 2)
        return fail(BN_ERR_INVALID_ARG, "couples_per_sweep must be in [0, 2^L / 2]");
    if (c.mode != BN_MODE_NONINTERACTING && c.mode != BN_MODE_CONCURRENT)
        return fail(BN_ERR_INVALID_ARG, "unknown mode %d", c.mode);
    if (c.objective != 0 && c.objective != BN_OBJECTIVE_BLUE && c.objective != BN_OBJECTIVE_LITERAL)
        return fail(BN_ERR_INVALID_ARG, "unknown objective %d", c.objective);
    if (c.schedule < BN_SCHEDULE_AUTO || c.schedule > BN_SCHEDULE_TENSOR)
        return fail(BN_ERR_INVALID_ARG, "unknown schedule %d", c.schedule);
    return BN_OK;
}

// Fill the geometry / stencil part of a problem descriptor.  The neighbourhood is every
// distinct pixel q != p of the torus within min-image distance r; offsets are the min-image
// representatives, sorted by squared distance (one class per distinct d^2).
void describe(const bn_config &c, int pair, bn::Problem &h)
{
    memset(&h, 0, sizeof h);
    h.W = c.width;
    h.H = c.height;
    h.P = c.width * c.height;
    h.L = log2_ceil(h.P);
    h.M = c.couples_per_sweep ? c.couples_per_sweep : ((1 << h.L) / 8 > 0 ? (1 << h.L) / 8 : 1);
    h.N = c.n_points;
    h.m = log2_ceil(c.n_points);
    h.g = c.generator_g ? c.generator_g : korobov_g(c.n_points);
    h.T = c.n_integrands;
    h.count_bytes = c.n_points <= 64 ? 1 : 2;
    h.row_bytes = (c.n_integrands * h.count_bytes + bn::kRowAlign - 1) / bn::kRowAlign *
                  bn::kRowAlign;
    h.radius = c.radius;
    h.mode = c.mode;
    h.objective = c.objective ? c.objective : BN_OBJECTIVE_BLUE;
    h.pair = (uint32_t)pair;
    h.seed_lo = (uint32_t)c.seed;
    h.seed_hi = (uint32_t)(c.seed >> 32);
    h.scale = 4.0f / ((float)c.n_points * (float)c.n_points);

    auto canonical = [](int d, int n) {
        int o = ((d % n) + n) % n;
        int rep = (2 * o <= n) ? o : o - n;
        return rep == d;
    };
    struct Off { int d2, dy, dx; };
    std::vector<Off> offs;
    const int r = c.radius;
    for (int dy = -r; dy <= r; ++dy)
        for (int dx = -r; dx <= r; ++dx) {
            if ((dx == 0 && dy == 0) || dx * dx + dy * dy > r * r) continue;
            if (!canonical(dx, c.width) || !canonical(dy, c.height)) continue;
            offs.push_back({dx * dx + dy * dy, dy, dx});
        }
    std::sort(offs.begin(), offs.end(), [](const Off &x, const Off &y) {
        if (x.d2 != y.d2) return x.d2 < y.d2;
        if (x.dy != y.dy) return x.dy < y.dy;
        return x.dx < y.dx;
    });
    h.n_off = (int)offs.size();
    int ncls = 0;
    for (int i = 0; i < h.n_off; ++i) {
        if (i == 0 || offs[i].d2 != offs[i - 1].d2) {
            h.d2[ncls] = offs[i].d2;
            h.w[ncls] = (float)std::exp(-(double)offs[i].d2 / ((double)c.sigma * c.sigma));
            h.cls_start[ncls] = i;
            ++ncls;
        }
        h.off[i] = (offs[i].dx & 0xFFFF) | (offs[i].dy << 16);
    }
    h.n_cls = ncls;
    h.cls_start[ncls] = h.n_off;
}

// carve the device arrays of one problem out of a slab (sizes only when base is null)
void carve(Slab &s, bn::Problem &h)
{
    h.counts = s.take<uint8_t>((size_t)h.P * h.row_bytes);
    h.U = s.take<uint32_t>((size_t)h.P * 2);
    h.sidx = s.take<int32_t>(h.P);
    h.perm = s.take<int32_t>((size_t)1 << h.L);
    h.perm_inv = s.take<int32_t>((size_t)1 << h.L);
    h.ha = s.take<int32_t>(h.T);
    h.hb = s.take<int32_t>(h.T);
    h.hC = s.take<int64_t>(h.T);
    h.owner = s.take<unsigned long long>((size_t)h.P * 2);
    h.log_dE = s.take<float>(h.M);
    h.log_flags = s.take<uint8_t>((size_t)h.M + 4);  // phase 2 reads aligned 4-byte words
    h.log_couples = s.take<int32_t>((size_t)h.M * 2);
    h.side_cls = s.take<int32_t>((size_t)h.M * 2 * bn::kMaxTsplit * bn::kMaxClasses);
    h.tc_npx = (h.W + 15) / 16;
    h.tc_npy = (h.H + 7) / 8;
    h.tc_cap = (16 + 2 * h.radius) * (8 + 2 * h.radius);
    h.tc_cnt = s.take<int32_t>((size_t)h.tc_npx * h.tc_npy);
    h.tc_list = s.take<int4>((size_t)h.tc_npx * h.tc_npy * h.tc_cap);
    h.ctr = s.take<long long>(4);
    h.stats = s.take<unsigned long long>(bn::kStatCount);
    h.esum = s.take<unsigned long long>(bn::kMaxClasses);
    h.energy_out = s.take<double>(1);
}

}  // namespace

// device bytes a sampler of this configuration holds (slab + staging), without allocating
int64_t bn::estimate_device_bytes(const bn_config &c)
{
    if (validate(c) != BN_OK) return -1;
    Slab sizing;
    size_t tc_extra = 0;  // a tensor-core plan's delta rows, tensor map and patch table
    for (int i = 0; i < c.n_pairs; ++i) {
        bn::Problem h;
        describe(c, i, h);
        carve(sizing, h);
        if (bn::tc_supported(h))
            tc_extra += bn::tc_delta_bytes(h) + (size_t)bn::tc_tensor_map_bytes() +
                        sizeof(int4) * (size_t)bn::tc_units_per_problem(h) + sizeof(bn::Problem);
    }
    return (int64_t)(sizing.used + 256 + sizeof(bn::Problem) * c.n_pairs + tc_extra +
                     sizeof(float) * (size_t)c.width * c.height * 2 * c.n_pairs + 4096);
}

namespace {

// Stream-ordered scratch, released on every return path
struct StreamScratch {
    void *ptr = nullptr;
    cudaStream_t st = nullptr;
    explicit StreamScratch(cudaStream_t s) : st(s) {}
    StreamScratch(const StreamScratch &) = delete;
    StreamScratch &operator=(const StreamScratch &) = delete;
    ~StreamScratch()
    {
        if (ptr) cudaFreeAsync(ptr, st);
    }
    cudaError_t alloc(size_t bytes) { return cudaMallocAsync(&ptr, bytes, st); }
    template <typename T>
    T *as() const
    {
        return static_cast<T *>(ptr);
    }
};

int check_pair(bn_sampler *s, int32_t pair)
{
    if (!s) return fail(BN_ERR_INVALID_ARG, "null sampler");
    if (pair < 0 || pair >= s->n_prob) return fail(BN_ERR_INVALID_ARG, "pair out of range");
    return BN_OK;
}

int set_device(const bn_sampler *s)
{
    int cur = -1;
    BN_CUDA(cudaGetDevice(&cur));
    if (cur != s->device) BN_CUDA(cudaSetDevice(s->device));
    return BN_OK;
}

// A bounded device-side wait that ran out leaves a sticky error in the problems' counters; the
// synchronous calls report it.  The sampler's stream must be synchronised.
int check_device_error(const bn_sampler *s)
{
    for (const auto &h : s->hprob) {
        unsigned long long err = 0;
        BN_CUDA(cudaMemcpy(&err, h.stats + bn::kStatError, sizeof err, cudaMemcpyDeviceToHost));
        if (err)
            return fail(BN_ERR_TIMEOUT, "a device-side wait ran out (code %llu); the sampler's "
                        "state is undefined, reset it", err);
    }
    return BN_OK;
}

// Build the execution plan of a problem list (grouped by count width, 1-byte group first).
// schedule: BN_SCHEDULE_*; the persistent schedule needs the radius-6 stencil on tiles of at
// least 13 x 13 for every problem.
int build_plan(const std::vector<bn::Problem> &hp, const bn::Problem *dprob, int schedule,
               const bn::PersistentShape *want, SweepPlan &pl)
{
    free_plan(pl);
    pl.n_prob = (int)hp.size();
    pl.max_M = 0;
    for (auto &h : hp) pl.max_M = h.M > pl.max_M ? h.M : pl.max_M;
    int dev = 0;
    BN_CUDA(cudaGetDevice(&dev));
    BN_CUDA(cudaDeviceGetAttribute(&pl.sms, cudaDevAttrMultiProcessorCount, dev));
    if (schedule == BN_SCHEDULE_TENSOR) {
        for (auto &h : hp)
            if (!bn::tc_supported(h))
                return fail(BN_ERR_INVALID_ARG, "the tensor-core schedule needs counts below "
                            "1024 (N <= 512), T N^2 <= 2^27 (exact centred products), radius "
                            "<= 8 and tile sides of at least 2 radius + 1");
        std::vector<int4> units;
        for (int i = 0; i < pl.n_prob; ++i)
            for (int pid = 0; pid < bn::tc_units_per_problem(hp[i]); ++pid)
                units.push_back(make_int4(i, pid, (pid % hp[i].tc_npx) * 16,
                                          (pid / hp[i].tc_npx) * 8));
        pl.tc_units = (int)units.size();
        pl.tc_rounds = false;
        for (auto &h : hp) pl.tc_rounds = pl.tc_rounds || bn::tc_rounds(h);
        BN_CUDA(bn::prepare_tc());
        pl.tcprob = hp;
        const size_t mb = (size_t)bn::tc_tensor_map_bytes();
        std::vector<char> maps((size_t)pl.n_prob * mb, 0);
        for (size_t i = 0; i < pl.tcprob.size(); ++i) {
            bn::Problem &h = pl.tcprob[i];
            void *d = nullptr;
            BN_CUDA(cudaMalloc(&d, bn::tc_delta_bytes(h)));
            pl.tc_bufs.push_back(d);
            h.tc_delta16 = static_cast<uint16_t *>(d);
            if (bn::encode_tc_tensor_map(h, maps.data() + i * mb) != cudaSuccess)
                return fail(BN_ERR_INVALID_ARG, "tensor map of the count planes could not be "
                            "encoded (%d x %d tile)", h.W, h.H);
        }
        BN_CUDA(cudaMalloc(&pl.d_tmaps, maps.size()));
        BN_CUDA(cudaMemcpy(pl.d_tmaps, maps.data(), maps.size(), cudaMemcpyHostToDevice));
        BN_CUDA(cudaMalloc(&pl.d_tcprob, sizeof(bn::Problem) * pl.tcprob.size()));
        BN_CUDA(cudaMemcpy(pl.d_tcprob, pl.tcprob.data(), sizeof(bn::Problem) * pl.tcprob.size(),
                           cudaMemcpyHostToDevice));
        BN_CUDA(cudaMalloc(&pl.d_tc_units, sizeof(int4) * units.size()));
        BN_CUDA(cudaMemcpy(pl.d_tc_units, units.data(), sizeof(int4) * units.size(),
                           cudaMemcpyHostToDevice));
        pl.tensor = true;
        pl.first[0] = 0;
        pl.count[0] = pl.n_prob;
        pl.first[1] = pl.count[1] = 0;
        return BN_OK;
    }
    bool ok = true;
    for (auto &h : hp) ok = ok && bn::persistent_supported(h);
    if (schedule == BN_SCHEDULE_PERSISTENT && !ok)
        return fail(BN_ERR_INVALID_ARG,
                    "the persistent schedule needs radius 6 and tiles of at least 13 x 13");
    pl.persistent = ok && schedule != BN_SCHEDULE_PLAIN;
    if (pl.persistent) {
        // requested shape, else the first instantiated shape that fits every problem
        std::vector<bn::PersistentShape> cands;
        if (want) cands.push_back(*want);
#define BN_CAND(BX, BY, NCW, SPW, MINB) cands.push_back(bn::PersistentShape{BX, BY, (NCW + 1) * 32, SPW, 0});
        BN_PERSISTENT_SHAPES(BN_CAND)
#undef BN_CAND
        bool found = false;
        for (auto &c : cands) {
            bool fits = true;
            for (auto &h : hp) fits = fits && bn::persistent_shape_fits(h, c);
            if (fits) {
                const int ts = want ? want->tsplit : 0;
                pl.shape = c;
                pl.shape.tsplit = ts;
                found = true;
                break;
            }
        }
        if (!found) {
            if (schedule == BN_SCHEDULE_PERSISTENT)
                return fail(BN_ERR_INVALID_ARG, "no persistent CTA shape fits these tiles");
            pl.persistent = false;
        }
    }
    for (int g = 0; g < 2; ++g) {
        pl.first[g] = pl.count[g] = 0;
        int f = -1;
        for (int i = 0; i < pl.n_prob; ++i)
            if (hp[i].count_bytes == g + 1) {
                if (f < 0) f = i;
                ++pl.count[g];
            }
        pl.first[g] = f < 0 ? 0 : f;
        for (int i = pl.first[g]; i < pl.first[g] + pl.count[g]; ++i)
            if (hp[i].count_bytes != g + 1)
                return fail(BN_ERR_INVALID_ARG, "internal: problems not grouped by count width");
    }
    if (!pl.persistent) return BN_OK;
    // default chunk split: enough work units to cover every SM twice
    int units1 = 0, min_chunks = 1 << 30;
    for (auto &h : hp) {
        units1 += bn::persistent_units_per_problem(h, pl.shape.bx, pl.shape.by, 1);
        const int nc = h.row_bytes / 128;
        min_chunks = nc < min_chunks ? nc : min_chunks;
    }
    if (pl.shape.tsplit <= 0) {
        int ts = (2 * pl.sms + units1 - 1) / units1;
        pl.shape.tsplit = ts;
    }
    if (pl.shape.tsplit > bn::kMaxTsplit) pl.shape.tsplit = bn::kMaxTsplit;
    if (pl.shape.tsplit > min_chunks) pl.shape.tsplit = min_chunks;
    if (pl.shape.tsplit < 1) pl.shape.tsplit = 1;
    std::vector<int> pre((size_t)4 * (pl.n_prob + 1), 0);
    for (int g = 0; g < 2; ++g) {
        int *us = pre.data() + (size_t)(2 * g) * (pl.n_prob + 1);
        int *cs = pre.data() + (size_t)(2 * g + 1) * (pl.n_prob + 1);
        for (int k = 0; k < pl.count[g]; ++k) {
            const bn::Problem &h = hp[pl.first[g] + k];
            us[k + 1] = us[k] + bn::persistent_units_per_problem(h, pl.shape.bx, pl.shape.by,
                                                                 pl.shape.tsplit);
            cs[k + 1] = cs[k] + h.M;
        }
        pl.total_units[g] = us[pl.count[g]];
        pl.total_couples[g] = cs[pl.count[g]];
    }
    BN_CUDA(cudaMalloc(&pl.d_prefix, sizeof(int) * pre.size()));
    BN_CUDA(cudaMemcpy(pl.d_prefix, pre.data(), sizeof(int) * pre.size(), cudaMemcpyHostToDevice));
    BN_CUDA(cudaMalloc(&pl.d_bar, sizeof(bn::GridBarrier)));
    BN_CUDA(cudaMalloc(&pl.d_work, 2 * sizeof(int)));
    (void)dprob;
    return BN_OK;
}

// A build that fails at any step (an allocation, a tensor-map encoding, an unsupported tile)
// leaves an empty plan that every sweep call refuses, never a half-built one whose kernels would
// be handed null device arrays.
int make_plan(const std::vector<bn::Problem> &hp, const bn::Problem *dprob, int schedule,
              const bn::PersistentShape *want, SweepPlan &pl)
{
    const int rc = build_plan(hp, dprob, schedule, want, pl);
    if (rc) {
        const std::string msg = g_error;
        free_plan(pl);
        cudaGetLastError();
        return fail(rc, "%s", msg.c_str());
    }
    pl.ready = true;
    return BN_OK;
}

constexpr int kItersPerLaunch = 500;

int plan_kind(const SweepPlan &pl)
{
    return pl.tensor ? BN_SCHEDULE_TENSOR
                     : (pl.persistent ? BN_SCHEDULE_PERSISTENT : BN_SCHEDULE_PLAIN);
}

// one pass of the plain or tensor-core schedule (three or five launches)
cudaError_t launch_pass(const SweepPlan &pl, const bn::SweepLaunch &sl, cudaStream_t st,
                        bn::KernelTimer *tm)
{
    if (!pl.tensor) return bn::launch_plain_sweep(sl, st, tm);
    const bn::TcLaunch tl{pl.d_tcprob, sl.n_prob, pl.max_M, pl.d_tc_units, pl.tc_units, pl.sms,
                          pl.d_tmaps, pl.tc_rounds};
    return bn::launch_tc_sweep(tl, st, tm);
}

int launches_per_pass(const SweepPlan &pl) { return pl.tensor ? 5 : 3; }  // lists+deltas, stencil,
                                                                           // finalize, resolve, commit

// Capture graph_passes passes of the plain or tensor-core schedule as one CUDA graph.  Every
// kernel reads the pass index and budget from device memory, so the graph replays.
int capture_plain(SweepPlan &pl, const bn::SweepLaunch &sl, int g)
{
    if (!pl.capture) BN_CUDA(cudaStreamCreateWithFlags(&pl.capture, cudaStreamNonBlocking));
    BN_CUDA(cudaStreamBeginCapture(pl.capture, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    const long long before = bn::launch_count();
    for (int k = 0; k < pl.graph_passes && e == cudaSuccess; ++k)
        e = launch_pass(pl, sl, pl.capture, nullptr);
    bn::note_launches(before - bn::launch_count());  // captured, not launched
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(pl.capture, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&pl.graph[g], graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        pl.graph[g] = nullptr;
        return fail(BN_ERR_CUDA, "capture of the sweep graph failed: %s",
                    cudaGetErrorString(e));
    }
    return BN_OK;
}

int run_plan(SweepPlan &pl, const bn::Problem *dprob, const std::vector<bn::Problem> &hp,
             int32_t n_sweeps, cudaStream_t st, bn::KernelTimer *tm, bool set_end = true)
{
    if (!pl.ready)
        return fail(BN_ERR_BAD_STATE, "no usable execution plan (a schedule change failed and "
                    "the default plan could not be rebuilt); reset or recreate the object");
    if (set_end) BN_CUDA(bn::launch_set_end(dprob, pl.n_prob, n_sweeps, 1, st));
    if (!pl.persistent) {
        // per-kernel timing needs the individual launches
        const bool graphs = pl.graph_passes > 0 && !(tm && tm->enabled);
        for (int g = 0; g < 2; ++g) {
            if (!pl.count[g]) continue;
            bn::SweepLaunch sl{dprob + pl.first[g], pl.count[g], pl.max_M, g + 1};
            int32_t k = 0;
            if (graphs && n_sweeps >= pl.graph_passes) {
                if (!pl.graph[g])
                    if (int rc = capture_plain(pl, sl, g)) return rc;
                for (; k + pl.graph_passes <= n_sweeps; k += pl.graph_passes)
                    BN_CUDA(cudaGraphLaunch(pl.graph[g], st));
                bn::note_launches((long long)launches_per_pass(pl) * pl.graph_passes *
                                  ((n_sweeps / pl.graph_passes)));
            }
            for (; k < n_sweeps; ++k) BN_CUDA(launch_pass(pl, sl, st, tm));
        }
        return BN_OK;
    }
    for (int g = 0; g < 2; ++g) {
        if (!pl.count[g]) continue;
        bn::PersistentArgs a{};
        a.probs = dprob + pl.first[g];
        a.n_prob = pl.count[g];
        a.unit_start = pl.d_prefix + (size_t)(2 * g) * (pl.n_prob + 1);
        a.couple_start = pl.d_prefix + (size_t)(2 * g + 1) * (pl.n_prob + 1);
        a.total_units = pl.total_units[g];
        a.total_couples = pl.total_couples[g];
        a.tsplit = pl.shape.tsplit;
        a.bar = pl.d_bar;
        a.work = pl.d_work;
        for (int32_t done = 0; done < n_sweeps; done += kItersPerLaunch) {
            a.n_iter = n_sweeps - done < kItersPerLaunch ? n_sweeps - done : kItersPerLaunch;
            BN_CUDA(cudaMemsetAsync(pl.d_bar, 0, sizeof(bn::GridBarrier), st));
            BN_CUDA(cudaMemsetAsync(pl.d_work, 0, 2 * sizeof(int), st));
            const bool timed = tm && tm->enabled;
            if (timed) tm->begin(bn::kKPersistent, st);
            cudaError_t e = bn::launch_persistent(a, pl.shape, g + 1, pl.sms, st);
            if (timed) tm->end(st);
            if (e != cudaSuccess)
                return fail(BN_ERR_CUDA, "persistent launch (%dx%d, %d threads) failed: %s",
                            pl.shape.bx, pl.shape.by, pl.shape.threads, cudaGetErrorString(e));
            BN_CUDA(bn::launch_fold_error(pl.d_bar, a.probs, a.n_prob, st));
        }
    }
    (void)hp;
    return BN_OK;
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------------------------
extern "C" {

const char *bn_last_error(void) { return g_error.c_str(); }

int bn_sampler_init(const bn_config *cfg, void *cuda_stream, bn_sampler **out)
{
    bn::TraceRange trace_("bn.sampler_init");
    if (!cfg || !out) return fail(BN_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    int rc = validate(*cfg);
    if (rc) return rc;
    auto *s = new bn_sampler();
    s->cfg = *cfg;
    s->stream = (cudaStream_t)cuda_stream;
    s->n_prob = cfg->n_pairs;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return fail(BN_ERR_CUDA, "no CUDA device");
    }
    s->hprob.resize(s->n_prob);
    Slab sizing;
    for (int i = 0; i < s->n_prob; ++i) {
        describe(*cfg, i, s->hprob[i]);
        carve(sizing, s->hprob[i]);
    }
    s->slab_bytes = sizing.used + 256;
    cudaError_t e = cudaMalloc(&s->slab, s->slab_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&s->dprob, sizeof(bn::Problem) * s->n_prob);
    if (e == cudaSuccess) e = cudaMallocHost(&s->h_energy, sizeof(double) * s->n_prob);
    if (e == cudaSuccess) e = cudaMallocHost(&s->h_pinned, sizeof(bn::Problem) * s->n_prob);
    const size_t shift_floats = (size_t)s->hprob[0].P * 2 * s->n_prob;
    if (e == cudaSuccess) e = cudaMalloc(&s->d_shifts, sizeof(float) * shift_floats);
    if (e == cudaSuccess) e = cudaMallocHost(&s->h_shifts, sizeof(float) * shift_floats);
    if (e != cudaSuccess) {
        const size_t bytes = s->slab_bytes;
        bn_sampler_destroy(s);
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? BN_ERR_OOM : BN_ERR_CUDA,
                    "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    Slab real;
    real.base = s->slab;
    real.cap = s->slab_bytes;
    for (int i = 0; i < s->n_prob; ++i) carve(real, s->hprob[i]);
    e = cudaMemcpyAsync(s->dprob, s->hprob.data(), sizeof(bn::Problem) * s->n_prob,
                        cudaMemcpyHostToDevice, s->stream);
    for (int i = 0; i < s->n_prob && e == cudaSuccess; ++i) {
        e = bn::launch_init_tables(s->dprob + i, s->hprob[i], s->stream);
        if (e == cudaSuccess) e = bn::launch_counts(s->dprob + i, s->hprob[i], s->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        bn_sampler_destroy(s);
        return fail(BN_ERR_CUDA, "initialisation failed: %s", cudaGetErrorString(e));
    }
    if (int rc2 = make_plan(s->hprob, s->dprob, cfg->schedule, nullptr, s->plan)) {
        std::string msg = g_error;
        bn_sampler_destroy(s);
        return fail(rc2, "%s", msg.c_str());
    }
    s->schedule = plan_kind(s->plan);
    *out = s;
    return BN_OK;
}

void bn_sampler_destroy(bn_sampler *s)
{
    if (!s) return;
    if (s->stream || s->slab) cudaStreamSynchronize(s->stream);
    if (s->slab) cudaFree(s->slab);
    if (s->dprob) cudaFree(s->dprob);
    if (s->h_energy) cudaFreeHost(s->h_energy);
    if (s->h_pinned) cudaFreeHost(s->h_pinned);
    if (s->d_shifts) cudaFree(s->d_shifts);
    if (s->h_shifts) cudaFreeHost(s->h_shifts);
    free_plan(s->plan);
    delete s;
}

int bn_get_info(bn_sampler *s, bn_info *info)
{
    if (!s || !info) return fail(BN_ERR_INVALID_ARG, "null argument");
    const bn::Problem &h = s->hprob[0];
    info->generator_g = h.g;
    info->log2_padded = h.L;
    info->couples = h.M;
    info->count_bytes = h.count_bytes;
    info->row_bytes = h.row_bytes;
    info->n_offsets = h.n_off;
    info->n_classes = h.n_cls;
    info->schedule = s->schedule;
    info->sweep = s->sweep;
    info->device_bytes = (int64_t)s->slab_bytes;
    info->reset_h2d_bytes = (int64_t)(sizeof(bn::Problem) * s->n_prob);
    return BN_OK;
}

int bn_evaluate_energy(bn_sampler *s, double *energy_per_pair)
{
    bn::TraceRange trace_("bn.evaluate_energy");
    if (!s || !energy_per_pair) return fail(BN_ERR_INVALID_ARG, "null argument");
    if (int rc = set_device(s)) return rc;
    BN_CUDA(bn::launch_energy(s->dprob, s->hprob.data(), s->n_prob, s->stream));
    for (int i = 0; i < s->n_prob; ++i)
        BN_CUDA(cudaMemcpyAsync(s->h_energy + i, s->hprob[i].energy_out, sizeof(double),
                                cudaMemcpyDeviceToHost, s->stream));
    BN_CUDA(cudaStreamSynchronize(s->stream));
    if (int rc = check_device_error(s)) return rc;
    for (int i = 0; i < s->n_prob; ++i) energy_per_pair[i] = s->h_energy[i];
    return BN_OK;
}

int bn_evaluate_energy_device(bn_sampler *s, double *energy_per_pair_device)
{
    if (!s || !energy_per_pair_device) return fail(BN_ERR_INVALID_ARG, "null argument");
    if (int rc = set_device(s)) return rc;
    BN_CUDA(bn::launch_energy(s->dprob, s->hprob.data(), s->n_prob, s->stream));
    BN_CUDA(bn::launch_energy_copy(s->dprob, s->n_prob, energy_per_pair_device, s->stream));
    return BN_OK;
}

int64_t bn_launch_counter(void) { return (int64_t)bn::launch_count(); }

int bn_selftest_wait_timeout(int32_t which, int64_t budget_cycles)
{
    if (which != 0 && which != 1) return fail(BN_ERR_INVALID_ARG, "which must be 0 or 1");
    if (budget_cycles < 1000 || budget_cycles > (1ll << 31))
        return fail(BN_ERR_INVALID_ARG, "budget_cycles must be in [1000, 2^31]");
    bn::GridBarrier *gb = nullptr;
    int *res = nullptr;
    int host = -1;
    cudaError_t e = cudaMalloc(&gb, sizeof *gb);
    if (e == cudaSuccess) e = cudaMalloc(&res, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(gb, 0, sizeof *gb);
    if (e == cudaSuccess) e = cudaMemset(res, 0xFF, sizeof(int));
    if (e == cudaSuccess) e = bn::launch_selftest_wait(which, budget_cycles, gb, res, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(&host, res, sizeof(int), cudaMemcpyDeviceToHost);
    if (gb) cudaFree(gb);
    if (res) cudaFree(res);
    if (e != cudaSuccess) return fail(BN_ERR_CUDA, "self-test launch failed: %s", cudaGetErrorString(e));
    if (host == 1) return fail(BN_ERR_TIMEOUT, "the wait ran out as expected");
    if (host == 0) return BN_OK;
    return fail(BN_ERR_BAD_STATE, "self-test produced no result");
}

}  // extern "C"

namespace {

int read_stats(const std::vector<bn::Problem> &hp, cudaStream_t st, bn_sweep_stats *stats)
{
    std::vector<unsigned long long> buf(bn::kStatCount);
    memset(stats, 0, sizeof *stats);
    for (const auto &h : hp) {
        BN_CUDA(cudaMemcpyAsync(buf.data(), h.stats, sizeof(unsigned long long) * bn::kStatCount,
                                cudaMemcpyDeviceToHost, st));
        BN_CUDA(cudaStreamSynchronize(st));
        stats->proposals += (int64_t)buf[bn::kStatValid];
        stats->improving += (int64_t)buf[bn::kStatImproving];
        stats->committed += (int64_t)buf[bn::kStatCommitted];
        stats->ties += (int64_t)buf[bn::kStatTies];
        stats->sweeps = (int64_t)buf[bn::kStatSweeps];
        if (buf[bn::kStatError])
            return fail(BN_ERR_TIMEOUT, "a device-side wait ran out (code %llu)",
                        (unsigned long long)buf[bn::kStatError]);
    }
    return BN_OK;
}

}  // namespace

extern "C" {

int bn_optimize_sweeps(bn_sampler *s, int32_t n_sweeps, bn_sweep_stats *stats)
{
    bn::TraceRange trace_("bn.optimize_sweeps");
    if (!s) return fail(BN_ERR_INVALID_ARG, "null sampler");
    if (n_sweeps < 0) return fail(BN_ERR_INVALID_ARG, "n_sweeps must be >= 0");
    if (int rc = set_device(s)) return rc;
    if (int rc = run_plan(s->plan, s->dprob, s->hprob, n_sweeps, s->stream, &s->timer)) return rc;
    s->sweep += n_sweeps;
    if (stats) return read_stats(s->hprob, s->stream, stats);
    return BN_OK;
}

int bn_fetch_shifts(bn_sampler *s, float *out, size_t n_floats, int out_is_device)
{
    if (!s || !out) return fail(BN_ERR_INVALID_ARG, "null argument");
    const size_t per = (size_t)s->hprob[0].P * 2;
    if (n_floats < per * s->n_prob) return fail(BN_ERR_INVALID_ARG, "output buffer too small");
    if (int rc = set_device(s)) return rc;
    float *dst = out_is_device ? out : s->d_shifts;
    for (int i = 0; i < s->n_prob; ++i)
        BN_CUDA(bn::launch_fetch_shifts(s->dprob + i, s->hprob[i], dst + per * i, s->stream));
    if (!out_is_device) {
        BN_CUDA(cudaMemcpyAsync(s->h_shifts, s->d_shifts, sizeof(float) * per * s->n_prob,
                                cudaMemcpyDeviceToHost, s->stream));
        BN_CUDA(cudaStreamSynchronize(s->stream));
        if (int rc = check_device_error(s)) return rc;
        memcpy(out, s->h_shifts, sizeof(float) * per * s->n_prob);
    }
    return BN_OK;
}

int bn_fetch_points(bn_sampler *s, int32_t pair, int32_t pixel, float *out, size_t n_floats)
{
    if (int rc = check_pair(s, pair)) return rc;
    const bn::Problem &h = s->hprob[pair];
    if (!out || pixel < 0 || pixel >= h.P || n_floats < (size_t)2 * h.N)
        return fail(BN_ERR_INVALID_ARG, "bad pixel or buffer");
    if (int rc = set_device(s)) return rc;
    StreamScratch tmp(s->stream);
    BN_CUDA(tmp.alloc(sizeof(float) * 2 * h.N));
    BN_CUDA(bn::launch_fetch_points(s->dprob + pair, h, pixel, tmp.as<float>(), s->stream));
    BN_CUDA(cudaMemcpyAsync(out, tmp.ptr, sizeof(float) * 2 * h.N, cudaMemcpyDeviceToHost,
                            s->stream));
    BN_CUDA(cudaStreamSynchronize(s->stream));
    return BN_OK;
}

int bn_evaluate_criterion(bn_sampler *s, int32_t pair, int32_t integrands, int32_t n_integrands,
                          const float *sigmas, int32_t n_sigma, double *rmse_out)
{
    bn::TraceRange trace_("bn.evaluate_criterion");
    if (int rc = check_pair(s, pair)) return rc;
    const bn::Problem &h = s->hprob[pair];
    if (!sigmas || !rmse_out) return fail(BN_ERR_INVALID_ARG, "null sigmas or output");
    if (integrands != BN_INTEGRANDS_HEAVISIDE && integrands != BN_INTEGRANDS_GAUSSIAN)
        return fail(BN_ERR_INVALID_ARG, "integrands must be BN_INTEGRANDS_HEAVISIDE or _GAUSSIAN");
    const int most = integrands == BN_INTEGRANDS_HEAVISIDE ? h.T : 4096;
    if (n_integrands < 1 || n_integrands > most)
        return fail(BN_ERR_INVALID_ARG, "n_integrands must be in [1, %d]", most);
    if (n_sigma < 1 || n_sigma > 64) return fail(BN_ERR_INVALID_ARG, "n_sigma must be in [1, 64]");
    for (int i = 0; i < n_sigma; ++i)
        if (!std::isfinite(sigmas[i]) || sigmas[i] > 4096.f)
            return fail(BN_ERR_INVALID_ARG, "sigma must be finite and at most 4096");
    if (int rc = set_device(s)) return rc;
    std::vector<double> sums(n_sigma, 0.0);
    BN_CUDA(bn::criterion_sums(s->dprob + pair, h, integrands, n_integrands, sigmas, n_sigma,
                               sums.data(), s->stream));
    if (int rc = check_device_error(s)) return rc;
    const double cells = (double)h.P * (double)n_integrands;
    for (int i = 0; i < n_sigma; ++i) rmse_out[i] = std::sqrt(sums[i] / cells);
    return BN_OK;
}

int bn_error_spectrum(bn_sampler *s, int32_t pair, int32_t integrands, int32_t n_integrands,
                      double *power_out, int64_t *counts_out, int32_t n_rings, int32_t *n_rings_out)
{
    bn::TraceRange trace_("bn.error_spectrum");
    if (int rc = check_pair(s, pair)) return rc;
    const bn::Problem &h = s->hprob[pair];
    if (h.W > 1024 || h.H > 1024)
        return fail(BN_ERR_INVALID_ARG, "the spectrum needs tile sides of at most 1024");
    const int need = bn::spectrum_rings(h.W, h.H, nullptr);
    if (n_rings_out) *n_rings_out = need;
    if (!power_out) return BN_OK;  // a query of the ring count
    if (n_rings < need) return fail(BN_ERR_INVALID_ARG, "the tile has %d rings", need);
    if (integrands != BN_INTEGRANDS_HEAVISIDE && integrands != BN_INTEGRANDS_GAUSSIAN)
        return fail(BN_ERR_INVALID_ARG, "integrands must be BN_INTEGRANDS_HEAVISIDE or _GAUSSIAN");
    const int most = integrands == BN_INTEGRANDS_HEAVISIDE ? h.T : 4096;
    if (n_integrands < 1 || n_integrands > most)
        return fail(BN_ERR_INVALID_ARG, "n_integrands must be in [1, %d]", most);
    if (int rc = set_device(s)) return rc;
    std::vector<double> sums(need, 0.0);
    BN_CUDA(bn::spectrum_sums(s->dprob + pair, h, integrands, n_integrands, sums.data(),
                              s->stream));
    if (int rc = check_device_error(s)) return rc;
    std::vector<int> ring;
    bn::spectrum_rings(h.W, h.H, &ring);
    std::vector<int64_t> cnt(need, 0);
    for (int r : ring) ++cnt[r];
    for (int b = 0; b < need; ++b) {
        power_out[b] = sums[b] / ((double)cnt[b] * (double)n_integrands);
        if (counts_out) counts_out[b] = cnt[b];
    }
    return BN_OK;
}

int bn_export_shift_table(bn_sampler *s, int32_t pair, uint32_t *out_device, size_t n_words)
{
    if (int rc = check_pair(s, pair)) return rc;
    const bn::Problem &h = s->hprob[pair];
    if (!out_device || n_words < (size_t)2 * h.P)
        return fail(BN_ERR_INVALID_ARG, "output buffer must hold 2 * width * height words");
    if (int rc = set_device(s)) return rc;
    BN_CUDA(bn::launch_shift_table(s->dprob + pair, h, out_device, s->stream));
    return BN_OK;
}

int bn_generate_samples(bn_sampler *s, int32_t x0, int32_t y0, int32_t width, int32_t height,
                        int32_t first_sample, int32_t n_samples, int32_t n_dims, float *out,
                        size_t n_floats, int32_t out_is_device)
{
    if (!s || !out) return fail(BN_ERR_INVALID_ARG, "null argument");
    const bn::Problem &h = s->hprob[0];
    if (width < 1 || height < 1 || n_samples < 1 || first_sample < 0 ||
        (long long)first_sample + n_samples > h.N)
        return fail(BN_ERR_INVALID_ARG, "need width, height, n_samples >= 1 and "
                    "0 <= first_sample, first_sample + n_samples <= n_points (%d)", h.N);
    if (n_dims < 1 || n_dims > 2 * s->n_prob)
        return fail(BN_ERR_INVALID_ARG, "n_dims must be in [1, 2 * n_pairs] (%d)", 2 * s->n_prob);
    const long long need = (long long)width * height * n_samples * n_dims;
    if (need > (1ll << 31)) return fail(BN_ERR_INVALID_ARG, "more than 2^31 values requested");
    if (n_floats < (size_t)need) return fail(BN_ERR_INVALID_ARG, "output buffer too small");
    if (int rc = set_device(s)) return rc;
    bn_sample_table tb;
    memset(&tb, 0, sizeof tb);
    tb.width = h.W;
    tb.height = h.H;
    tb.n_pairs = s->n_prob;
    tb.log2_points = h.m;
    tb.generator_g = h.g;
    StreamScratch table_buf(s->stream), out_buf(s->stream);
    BN_CUDA(table_buf.alloc(sizeof(uint32_t) * 2 * h.P * s->n_prob));
    if (!out_is_device) BN_CUDA(out_buf.alloc(sizeof(float) * need));
    uint32_t *tables = table_buf.as<uint32_t>();
    float *dout = out_is_device ? out : out_buf.as<float>();
    for (int i = 0; i < s->n_prob; ++i) {
        BN_CUDA(bn::launch_shift_table(s->dprob + i, h, tables + (size_t)2 * h.P * i, s->stream));
        tb.shifts[i] = tables + (size_t)2 * h.P * i;
    }
    BN_CUDA(bn::launch_samples(tb, x0, y0, width, height, first_sample, n_samples, n_dims, dout,
                               s->stream));
    if (!out_is_device) {
        BN_CUDA(cudaMemcpyAsync(out, dout, sizeof(float) * need, cudaMemcpyDeviceToHost,
                                s->stream));
        BN_CUDA(cudaStreamSynchronize(s->stream));
    }
    return BN_OK;
}

int bn_fetch_counts(bn_sampler *s, int32_t pair, int32_t *out, size_t n)
{
    if (int rc = check_pair(s, pair)) return rc;
    const bn::Problem &h = s->hprob[pair];
    const size_t need = (size_t)h.P * h.T;
    if (!out || n < need) return fail(BN_ERR_INVALID_ARG, "output buffer too small");
    if (int rc = set_device(s)) return rc;
    StreamScratch tmp(s->stream);
    BN_CUDA(tmp.alloc(sizeof(int32_t) * need));
    BN_CUDA(bn::launch_unpack_counts(s->dprob + pair, h, tmp.as<int32_t>(), s->stream));
    BN_CUDA(cudaMemcpyAsync(out, tmp.ptr, sizeof(int32_t) * need, cudaMemcpyDeviceToHost,
                            s->stream));
    BN_CUDA(cudaStreamSynchronize(s->stream));
    return BN_OK;
}

int bn_fetch_integrands(bn_sampler *s, int32_t pair, int32_t *a, int32_t *b, int64_t *C,
                        size_t T)
{
    if (int rc = check_pair(s, pair)) return rc;
    const bn::Problem &h = s->hprob[pair];
    if (T < (size_t)h.T) return fail(BN_ERR_INVALID_ARG, "output buffer too small");
    if (int rc = set_device(s)) return rc;
    if (a) BN_CUDA(cudaMemcpyAsync(a, h.ha, sizeof(int32_t) * h.T, cudaMemcpyDeviceToHost, s->stream));
    if (b) BN_CUDA(cudaMemcpyAsync(b, h.hb, sizeof(int32_t) * h.T, cudaMemcpyDeviceToHost, s->stream));
    if (C) BN_CUDA(cudaMemcpyAsync(C, h.hC, sizeof(int64_t) * h.T, cudaMemcpyDeviceToHost, s->stream));
    BN_CUDA(cudaStreamSynchronize(s->stream));
    return BN_OK;
}

int bn_fetch_permutation(bn_sampler *s, int32_t pair, int32_t *out, size_t n)
{
    if (int rc = check_pair(s, pair)) return rc;
    const bn::Problem &h = s->hprob[pair];
    if (!out || n < ((size_t)1 << h.L)) return fail(BN_ERR_INVALID_ARG, "output buffer too small");
    if (int rc = set_device(s)) return rc;
    BN_CUDA(cudaMemcpyAsync(out, h.perm, sizeof(int32_t) << h.L, cudaMemcpyDeviceToHost,
                            s->stream));
    BN_CUDA(cudaStreamSynchronize(s->stream));
    return BN_OK;
}

int bn_fetch_sweep_log(bn_sampler *s, int32_t pair, float *dE, uint8_t *flags,
                       int32_t *couples, size_t cap)
{
    if (int rc = check_pair(s, pair)) return rc;
    const bn::Problem &h = s->hprob[pair];
    if (cap < (size_t)h.M) return fail(BN_ERR_INVALID_ARG, "cap < couples per pass");
    if (int rc = set_device(s)) return rc;
    if (dE) BN_CUDA(cudaMemcpyAsync(dE, h.log_dE, sizeof(float) * h.M, cudaMemcpyDeviceToHost, s->stream));
    if (flags) BN_CUDA(cudaMemcpyAsync(flags, h.log_flags, h.M, cudaMemcpyDeviceToHost, s->stream));
    if (couples)
        BN_CUDA(cudaMemcpyAsync(couples, h.log_couples, sizeof(int32_t) * 2 * h.M,
                                cudaMemcpyDeviceToHost, s->stream));
    BN_CUDA(cudaStreamSynchronize(s->stream));
    return BN_OK;
}

int bn_get_state(bn_sampler *s, int64_t *sweep, int32_t *shift_index, size_t n)
{
    if (!s) return fail(BN_ERR_INVALID_ARG, "null sampler");
    const size_t P = (size_t)s->hprob[0].P;
    if (shift_index && n < P * s->n_prob) return fail(BN_ERR_INVALID_ARG, "buffer too small");
    if (int rc = set_device(s)) return rc;
    if (shift_index)
        for (int i = 0; i < s->n_prob; ++i)
            BN_CUDA(cudaMemcpyAsync(shift_index + P * i, s->hprob[i].sidx, sizeof(int32_t) * P,
                                    cudaMemcpyDeviceToHost, s->stream));
    BN_CUDA(cudaStreamSynchronize(s->stream));
    if (int rc = check_device_error(s)) return rc;
    if (sweep) *sweep = s->sweep;
    return BN_OK;
}

int bn_set_state(bn_sampler *s, int64_t sweep, const int32_t *shift_index, size_t n)
{
    if (!s || !shift_index) return fail(BN_ERR_INVALID_ARG, "null argument");
    const size_t P = (size_t)s->hprob[0].P;
    if (n < P * s->n_prob || sweep < 0) return fail(BN_ERR_INVALID_ARG, "bad state");
    // the shift index must be a permutation of the pixels
    std::vector<char> seen(P);
    for (int i = 0; i < s->n_prob; ++i) {
        std::fill(seen.begin(), seen.end(), 0);
        for (size_t p = 0; p < P; ++p) {
            int32_t v = shift_index[P * i + p];
            if (v < 0 || (size_t)v >= P || seen[v])
                return fail(BN_ERR_INVALID_ARG, "shift_index of pair %d is not a permutation", i);
            seen[v] = 1;
        }
    }
    if (int rc = set_device(s)) return rc;
    for (int i = 0; i < s->n_prob; ++i) {
        BN_CUDA(cudaMemcpyAsync(s->hprob[i].sidx, shift_index + P * i, sizeof(int32_t) * P,
                                cudaMemcpyHostToDevice, s->stream));
        BN_CUDA(cudaMemcpyAsync(s->hprob[i].ctr, &sweep, sizeof(int64_t),
                                cudaMemcpyHostToDevice, s->stream));
        BN_CUDA(bn::launch_counts(s->dprob + i, s->hprob[i], s->stream));
    }
    BN_CUDA(cudaStreamSynchronize(s->stream));
    s->sweep = sweep;
    return BN_OK;
}

int bn_sampler_reset(bn_sampler *s, uint64_t seed)
{
    bn::TraceRange trace_("bn.sampler_reset");
    if (!s) return fail(BN_ERR_INVALID_ARG, "null sampler");
    if (int rc = set_device(s)) return rc;
    s->cfg.seed = seed;
    for (int i = 0; i < s->n_prob; ++i) {
        s->hprob[i].seed_lo = (uint32_t)seed;
        s->hprob[i].seed_hi = (uint32_t)(seed >> 32);
    }
    // the previous copy out of the pinned staging must be complete before it is rewritten
    BN_CUDA(cudaStreamSynchronize(s->stream));
    memcpy(s->h_pinned, s->hprob.data(), sizeof(bn::Problem) * s->n_prob);
    BN_CUDA(cudaMemcpyAsync(s->dprob, s->h_pinned, sizeof(bn::Problem) * s->n_prob,
                            cudaMemcpyHostToDevice, s->stream));
    for (int i = 0; i < s->n_prob; ++i) {
        BN_CUDA(bn::launch_init_tables(s->dprob + i, s->hprob[i], s->stream));
        BN_CUDA(bn::launch_counts(s->dprob + i, s->hprob[i], s->stream));
    }
    s->sweep = 0;
    return BN_OK;
}

int bn_set_kernel_timing(bn_sampler *s, int enable)
{
    if (!s) return fail(BN_ERR_INVALID_ARG, "null sampler");
    s->timer.enabled = enable != 0;
    s->timer.detail = enable >= 2;
    return BN_OK;
}

int bn_kernel_times(bn_sampler *s, bn_kernel_time *out, int32_t cap, int32_t *n_out)
{
    if (!s || !out || !n_out) return fail(BN_ERR_INVALID_ARG, "null argument");
    BN_CUDA(s->timer.collect());
    int n = 0;
    for (int k = 0; k < bn::kKindCount && n < cap; ++k) {
        if (!s->timer.launches[k]) continue;
        memset(&out[n], 0, sizeof out[n]);
        strncpy(out[n].name, bn::kKernelNames[k], sizeof out[n].name - 1);
        out[n].launches = s->timer.launches[k];
        out[n].total_ms = s->timer.ms[k];
        ++n;
    }
    *n_out = n;
    s->timer.reset();
    return BN_OK;
}

}  // extern "C"

static int set_schedule_common(const std::vector<bn::Problem> &hp, const bn::Problem *dprob,
                               const bn_schedule *sc, SweepPlan &plan)
{
    if (!sc) return fail(BN_ERR_INVALID_ARG, "null schedule");
    if (sc->kind != BN_SCHEDULE_PLAIN && sc->kind != BN_SCHEDULE_PERSISTENT &&
        sc->kind != BN_SCHEDULE_AUTO && sc->kind != BN_SCHEDULE_TENSOR)
        return fail(BN_ERR_INVALID_ARG, "unknown schedule kind %d", sc->kind);
    bn::PersistentShape shape{sc->block_x, sc->block_y, sc->threads, sc->slots_per_warp,
                              sc->tsplit};
    bool known = false;
#define BN_KNOWN(BX, BY, NCW, SPW, MINB)                                                      \
    known = known || (shape.bx == BX && shape.by == BY && shape.threads == (NCW + 1) * 32 &&     \
                      shape.spw == SPW);
    BN_PERSISTENT_SHAPES(BN_KNOWN)
#undef BN_KNOWN
    const bool want_shape = (sc->kind == BN_SCHEDULE_PERSISTENT || sc->kind == BN_SCHEDULE_AUTO) &&
                            sc->block_x > 0;
    if (want_shape && !known)
        return fail(BN_ERR_INVALID_ARG, "no kernel instantiated for block %dx%d, %d threads, %d "
                    "slots per warp", sc->block_x, sc->block_y, sc->threads, sc->slots_per_warp);
    const int rc = make_plan(hp, dprob, sc->kind, want_shape ? &shape : nullptr, plan);
    if (rc) {  // the previous plan is gone: leave the default one so the object stays usable
        const std::string msg = g_error;
        cudaGetLastError();
        if (make_plan(hp, dprob, BN_SCHEDULE_AUTO, nullptr, plan) != BN_OK)
            return fail(rc, "%s (and the default plan could not be rebuilt: %s; sweeps now "
                        "return BN_ERR_BAD_STATE)", msg.c_str(), g_error.c_str());
        return fail(rc, "%s", msg.c_str());
    }
    return BN_OK;
}

static void get_schedule_common(const SweepPlan &pl, bn_schedule *out)
{
    out->kind = plan_kind(pl);
    out->block_x = pl.shape.bx;
    out->block_y = pl.shape.by;
    out->threads = pl.shape.threads;
    out->slots_per_warp = pl.shape.spw;
    out->tsplit = pl.shape.tsplit;
}

// ---- autotuner: choose the execution schedule of a problem list by timing trial passes -----
// Trials run on a scratch copy of the members' device state (one device-to-device copy of each
// member's slab, descriptors rebased onto it), so the caller's tiles are untouched; since every
// schedule produces bit-identical results, the choice only affects speed.  Choices are cached
// per process by workload signature and, when BN_AUTOTUNE_CACHE names a file, in that file.
namespace {

std::mutex g_tune_mu;
std::map<std::string, bn_schedule> g_tune_cache;
bool g_tune_file_loaded = false;

std::string tune_key(const std::vector<bn::Problem> &hp, int sms)
{
    std::string k = "sm" + std::to_string(sms);
    for (const auto &h : hp)
        k += "|" + std::to_string(h.W) + "x" + std::to_string(h.H) + "n" + std::to_string(h.N) +
             "t" + std::to_string(h.T) + "m" + std::to_string(h.M) + "r" + std::to_string(h.radius);
    return k;
}

void tune_file_load()
{
    if (g_tune_file_loaded) return;
    g_tune_file_loaded = true;
    const char *path = std::getenv("BN_AUTOTUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    char key[8192];
    bn_schedule sc{};
    while (std::fscanf(f, "%8191s %d %d %d %d %d %d", key, &sc.kind, &sc.block_x, &sc.block_y,
                       &sc.threads, &sc.slots_per_warp, &sc.tsplit) == 7)
        g_tune_cache[key] = sc;
    std::fclose(f);
}

void tune_file_store(const std::string &key, const bn_schedule &sc)
{
    const char *path = std::getenv("BN_AUTOTUNE_CACHE");
    if (!path || key.size() > 8000) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s %d %d %d %d %d %d\n", key.c_str(), sc.kind, sc.block_x, sc.block_y,
                 sc.threads, sc.slots_per_warp, sc.tsplit);
    std::fclose(f);
}

void rebase(bn::Problem &h, const char *from, char *to)
{
    auto mv = [&](auto *&p) {
        if (p) p = reinterpret_cast<std::remove_reference_t<decltype(p)>>(
                   to + (reinterpret_cast<const char *>(p) - from));
    };
    mv(h.counts); mv(h.U); mv(h.sidx); mv(h.perm); mv(h.perm_inv); mv(h.ha); mv(h.hb);
    mv(h.hC); mv(h.owner); mv(h.log_dE); mv(h.log_flags); mv(h.log_couples);
    mv(h.side_cls); mv(h.tc_cnt); mv(h.tc_list); mv(h.ctr); mv(h.stats); mv(h.esum);
    mv(h.energy_out);
}

// Time every candidate schedule on a scratch copy of the members; returns the fastest.
int autotune(const std::vector<bn_sampler *> &members, int32_t trial_sweeps, cudaStream_t st,
             bn_schedule *best)
{
    // scratch copy, problems grouped by count width as in a batch
    std::vector<char *> clones(members.size(), nullptr);
    std::vector<bn::Problem> hp;
    bn::Problem *dp = nullptr;
    SweepPlan plan;
    int rc = BN_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&]() {
        cudaStreamSynchronize(st);
        for (char *c : clones)
            if (c) cudaFree(c);
        if (dp) cudaFree(dp);
        free_plan(plan);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    for (size_t i = 0; i < members.size(); ++i) {
        cudaError_t e = cudaMalloc(&clones[i], members[i]->slab_bytes);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(clones[i], members[i]->slab, members[i]->slab_bytes,
                                cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) {
            cleanup();
            return fail(e == cudaErrorMemoryAllocation ? BN_ERR_OOM : BN_ERR_CUDA,
                        "autotune scratch copy failed: %s", cudaGetErrorString(e));
        }
    }
    for (int cb = 1; cb <= 2; ++cb)
        for (size_t i = 0; i < members.size(); ++i)
            for (auto h : members[i]->hprob)
                if (h.count_bytes == cb) {
                    rebase(h, members[i]->slab, clones[i]);
                    hp.push_back(h);
                }
    cudaError_t e = cudaMalloc(&dp, sizeof(bn::Problem) * hp.size());
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dp, hp.data(), sizeof(bn::Problem) * hp.size(),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cleanup();
        return fail(BN_ERR_CUDA, "autotune setup failed: %s", cudaGetErrorString(e));
    }
    std::vector<bn_schedule> cands;
#define BN_CAND(BX, BY, NCW, SPW, MINB)                                                        \
    for (int ts = 1; ts <= 2; ++ts) cands.push_back(bn_schedule{BN_SCHEDULE_PERSISTENT, BX, BY,   \
                                                                (NCW + 1) * 32, SPW, ts});
    BN_PERSISTENT_SHAPES(BN_CAND)
#undef BN_CAND
    cands.push_back(bn_schedule{BN_SCHEDULE_TENSOR, 0, 0, 0, 0, 0});
    cands.push_back(bn_schedule{BN_SCHEDULE_PLAIN, 0, 0, 0, 0, 0});
    float best_ms = -1.f;
    for (const auto &c : cands) {
        bn::PersistentShape shape{c.block_x, c.block_y, c.threads, c.slots_per_warp, c.tsplit};
        bool fits = c.kind == BN_SCHEDULE_PLAIN;
        if (c.kind == BN_SCHEDULE_TENSOR) {
            fits = true;
            for (const auto &h : hp) fits = fits && bn::tc_supported(h);
        } else if (!fits) {
            fits = true;
            for (const auto &h : hp)
                fits = fits && bn::persistent_shape_fits(h, shape) && h.row_bytes / 128 >= c.tsplit;
        }
        if (!fits) continue;
        if (c.kind == BN_SCHEDULE_PLAIN && best_ms >= 0.f) continue;  // plain only as fallback
        if ((rc = make_plan(hp, dp, c.kind, c.kind == BN_SCHEDULE_PERSISTENT ? &shape : nullptr,
                            plan))) {
            if (c.kind != BN_SCHEDULE_TENSOR) break;
            // the tensor-core plan could not allocate its delta rows: not a candidate here
            cudaGetLastError();
            free_plan(plan);
            rc = BN_OK;
            continue;
        }
        if ((rc = run_plan(plan, dp, hp, 2, st, nullptr))) break;  // warm
        cudaEventRecord(e0, st);
        if ((rc = run_plan(plan, dp, hp, trial_sweeps, st, nullptr))) break;
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            rc = fail(BN_ERR_CUDA, "autotune trial failed: %s", cudaGetErrorString(e));
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (best_ms < 0.f || ms < best_ms) {
            best_ms = ms;
            *best = c;
        }
    }
    cleanup();
    if (rc) return rc;
    if (best_ms < 0.f) return fail(BN_ERR_BAD_STATE, "autotune found no runnable schedule");
    return BN_OK;
}

int autotune_entry(const std::vector<bn_sampler *> &members, const std::vector<bn::Problem> &hp,
                   const bn::Problem *dprob, cudaStream_t st, int32_t trial_sweeps,
                   SweepPlan &plan, bn_schedule *chosen)
{
    if (trial_sweeps < 1 || trial_sweeps > 10000)
        return fail(BN_ERR_INVALID_ARG, "trial_sweeps must be in [1, 10000]");
    int dev = 0, sms = 0;
    BN_CUDA(cudaGetDevice(&dev));
    BN_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const std::string key = tune_key(hp, sms);
    bn_schedule best{};
    bool hit = false;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_file_load();
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            best = it->second;
            hit = true;
        }
    }
    // a cached choice that no longer names a usable schedule (a cache file written by another
    // build) is tuned again
    if (hit && set_schedule_common(hp, dprob, &best, plan) != BN_OK) hit = false;
    if (!hit) {
        for (auto *m : members) BN_CUDA(cudaStreamSynchronize(m->stream));
        if (int rc = autotune(members, trial_sweeps, st, &best)) return rc;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tune_cache[key] = best;
            tune_file_store(key, best);
        }
        if (int rc = set_schedule_common(hp, dprob, &best, plan)) return rc;
    }
    if (chosen) *chosen = best;
    return BN_OK;
}

// work that a member later enqueues on its own stream starts after the batch's last sweep call
int order_members_after(bn_batch *b)
{
    BN_CUDA(cudaEventRecord(b->done, b->stream));
    for (auto *m : b->members)
        if (m->stream != b->stream) BN_CUDA(cudaStreamWaitEvent(m->stream, b->done, 0));
    return BN_OK;
}

}  // namespace

extern "C" {

int bn_sampler_autotune(bn_sampler *s, int32_t trial_sweeps, bn_schedule *chosen)
{
    if (!s) return fail(BN_ERR_INVALID_ARG, "null sampler");
    if (int rc = set_device(s)) return rc;
    if (int rc = autotune_entry({s}, s->hprob, s->dprob, s->stream, trial_sweeps, s->plan, chosen))
        return rc;
    s->schedule = plan_kind(s->plan);
    return BN_OK;
}

int bn_sampler_set_schedule(bn_sampler *s, const bn_schedule *sc)
{
    if (!s) return fail(BN_ERR_INVALID_ARG, "null sampler");
    if (int rc = set_device(s)) return rc;
    BN_CUDA(cudaStreamSynchronize(s->stream));
    const int rc = set_schedule_common(s->hprob, s->dprob, sc, s->plan);
    s->schedule = plan_kind(s->plan);
    return rc;
}

int bn_sampler_get_schedule(bn_sampler *s, bn_schedule *out)
{
    if (!s || !out) return fail(BN_ERR_INVALID_ARG, "null argument");
    get_schedule_common(s->plan, out);
    return BN_OK;
}

int bn_batch_set_schedule(bn_batch *b, const bn_schedule *sc)
{
    if (!b) return fail(BN_ERR_INVALID_ARG, "null batch");
    BN_CUDA(cudaStreamSynchronize(b->stream));
    return set_schedule_common(b->all, b->dprob, sc, b->plan);
}

int bn_batch_optimize_each(bn_batch *b, const int32_t *n_sweeps_per_member,
                           bn_sweep_stats *stats)
{
    bn::TraceRange trace_("bn.batch_optimize_each");
    if (!b || !n_sweeps_per_member) return fail(BN_ERR_INVALID_ARG, "null argument");
    int32_t most = 0;
    for (size_t i = 0; i < b->members.size(); ++i) {
        if (n_sweeps_per_member[i] < 0) return fail(BN_ERR_INVALID_ARG, "negative pass count");
        most = n_sweeps_per_member[i] > most ? n_sweeps_per_member[i] : most;
    }
    for (auto *m : b->members)
        if (m->stream != b->stream) BN_CUDA(cudaStreamSynchronize(m->stream));
    // the pinned staging may still feed the previous call's copy
    BN_CUDA(cudaStreamSynchronize(b->stream));
    for (int i = 0; i < b->n_prob; ++i) b->h_ends[i] = n_sweeps_per_member[b->member_of[i]];
    BN_CUDA(cudaMemcpyAsync(b->d_ends, b->h_ends, sizeof(int) * b->n_prob,
                            cudaMemcpyHostToDevice, b->stream));
    BN_CUDA(bn::launch_set_ends(b->dprob, b->n_prob, b->d_ends, 1, b->stream));
    if (int rc = run_plan(b->plan, b->dprob, b->all, most, b->stream, b->timer, false)) return rc;
    if (int rc = order_members_after(b)) return rc;
    for (size_t i = 0; i < b->members.size(); ++i) b->members[i]->sweep += n_sweeps_per_member[i];
    if (stats) return read_stats(b->all, b->stream, stats);
    return BN_OK;
}

int bn_batch_autotune(bn_batch *b, int32_t trial_sweeps, bn_schedule *chosen)
{
    if (!b) return fail(BN_ERR_INVALID_ARG, "null batch");
    return autotune_entry(b->members, b->all, b->dprob, b->stream, trial_sweeps, b->plan, chosen);
}

int bn_sampler_set_graph_passes(bn_sampler *s, int32_t passes)
{
    if (!s || passes < 0 || passes > 4096)
        return fail(BN_ERR_INVALID_ARG, "passes per graph must be in [0, 4096]");
    if (int rc = set_device(s)) return rc;
    BN_CUDA(cudaStreamSynchronize(s->stream));
    free_graphs(s->plan);
    s->plan.graph_passes = passes;
    return BN_OK;
}

int bn_batch_set_graph_passes(bn_batch *b, int32_t passes)
{
    if (!b || passes < 0 || passes > 4096)
        return fail(BN_ERR_INVALID_ARG, "passes per graph must be in [0, 4096]");
    BN_CUDA(cudaStreamSynchronize(b->stream));
    free_graphs(b->plan);
    b->plan.graph_passes = passes;
    return BN_OK;
}

int bn_batch_get_schedule(bn_batch *b, bn_schedule *out)
{
    if (!b || !out) return fail(BN_ERR_INVALID_ARG, "null argument");
    get_schedule_common(b->plan, out);
    return BN_OK;
}

// ---- batches ---------------------------------------------------------------------------------
int bn_batch_create(bn_sampler *const *samplers, int32_t n, void *cuda_stream, bn_batch **out)
{
    return bn::batch_create_as(samplers, n, cuda_stream, BN_SCHEDULE_AUTO, out);
}

}  // extern "C"

int bn::batch_create_as(bn_sampler *const *samplers, int32_t n, void *cuda_stream, int schedule,
                        bn_batch **out)
{
    bn::TraceRange trace_("bn.batch_create");
    if (!samplers || n <= 0 || !out) return fail(BN_ERR_INVALID_ARG, "bad batch arguments");
    *out = nullptr;
    auto *b = new bn_batch();
    b->stream = (cudaStream_t)cuda_stream;
    std::vector<bn::Problem> all;
    for (int cb = 1; cb <= 2; ++cb)  // equal count widths contiguous
        for (int i = 0; i < n; ++i) {
            if (!samplers[i]) {
                delete b;
                return fail(BN_ERR_INVALID_ARG, "null sampler in batch");
            }
            for (auto &h : samplers[i]->hprob)
                if (h.count_bytes == cb) {
                    all.push_back(h);
                    b->member_of.push_back(i);
                }
        }
    for (int i = 0; i < n; ++i) b->members.push_back(samplers[i]);
    b->timer = &samplers[0]->timer;
    b->n_prob = (int)all.size();
    for (auto &h : all) b->max_M = h.M > b->max_M ? h.M : b->max_M;
    cudaError_t e = cudaMalloc(&b->dprob, sizeof(bn::Problem) * all.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(b->dprob, all.data(), sizeof(bn::Problem) * all.size(),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_ends, sizeof(int) * all.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->d_ends, sizeof(int) * all.size());
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        bn_batch_destroy(b);
        return fail(BN_ERR_CUDA, "batch allocation failed: %s", cudaGetErrorString(e));
    }
    int sched = schedule;
    if (sched == BN_SCHEDULE_AUTO) {  // derived from the members' configured schedules
        bool all_tensor = true;
        for (int i = 0; i < n; ++i) {
            if (samplers[i]->cfg.schedule == BN_SCHEDULE_PLAIN) sched = BN_SCHEDULE_PLAIN;
            all_tensor = all_tensor && samplers[i]->cfg.schedule == BN_SCHEDULE_TENSOR;
        }
        if (all_tensor && sched == BN_SCHEDULE_AUTO) sched = BN_SCHEDULE_TENSOR;
    }
    b->all = all;
    if (int rc = make_plan(b->all, b->dprob, sched, nullptr, b->plan)) {
        std::string msg = g_error;
        bn_batch_destroy(b);
        return fail(rc, "%s", msg.c_str());
    }
    *out = b;
    return BN_OK;
}

int bn::tune_schedule(bn_sampler *s, int32_t trial_sweeps, bn_schedule *best)
{
    if (!s || !best) return fail(BN_ERR_INVALID_ARG, "null argument");
    if (trial_sweeps < 1 || trial_sweeps > 10000)
        return fail(BN_ERR_INVALID_ARG, "trial_sweeps must be in [1, 10000]");
    if (int rc = set_device(s)) return rc;
    BN_CUDA(cudaStreamSynchronize(s->stream));
    return autotune({s}, trial_sweeps, s->stream, best);
}

bool bn::tensor_capable(const bn_sampler *s)
{
    if (!s) return false;
    for (const auto &h : s->hprob)
        if (!bn::tc_supported(h)) return false;
    return true;
}

extern "C" {

int bn_batch_optimize(bn_batch *b, int32_t n_sweeps, bn_sweep_stats *stats)
{
    bn::TraceRange trace_("bn.batch_optimize");
    if (!b || n_sweeps < 0) return fail(BN_ERR_INVALID_ARG, "bad batch call");
    // order the batch after every member's pending work
    for (auto *m : b->members) {
        if (m->stream == b->stream) continue;
        BN_CUDA(cudaStreamSynchronize(m->stream));
    }
    if (int rc = run_plan(b->plan, b->dprob, b->all, n_sweeps, b->stream, b->timer)) return rc;
    if (int rc = order_members_after(b)) return rc;
    for (auto *m : b->members) m->sweep += n_sweeps;
    if (stats) return read_stats(b->all, b->stream, stats);
    return BN_OK;
}

void bn_batch_destroy(bn_batch *b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    if (b->dprob) cudaFree(b->dprob);
    if (b->h_ends) cudaFreeHost(b->h_ends);
    if (b->d_ends) cudaFree(b->d_ends);
    if (b->done) cudaEventDestroy(b->done);
    free_plan(b->plan);
    delete b;
}

}  // extern "C"
