// qieo_api.cu -- host side of the C ABI declared in include/qieo.h.
//
// An instance owns one device allocation holding the qubit state, the two allele planes,
// the items (packed and wide form), the best row, the row accumulators and counters, the
// elite key and index, the grid-barrier words and the per-generation records. qieo_run
// enqueues one fused generation kernel per generation plus one final CIP launch, chained
// with programmatic dependent launch (each kernel's prologue overlaps the previous kernel's
// tail) and replayed from a cached CUDA graph when a run length repeats; with
// QIEO_FLAG_COOPERATIVE the whole run is one cooperative kernel whose blocks meet at a
// bounded grid barrier after each generation. With elite_on_host it copies the fitness array to the
// host after each generation, picks the elite there and records it with a one-block
// kernel (the host DetermineElite variant the paper recommends, Sec. III-C, Sec. VII P4).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <unordered_map>
#include <tuple>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/qieo.h"
#include "qieo_kernels.cuh"

namespace {

thread_local std::string g_last_error;

qieo_status fail(qieo_status st, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
qieo_status fail(qieo_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

#define CUDA_TRY(expr)                                                                     \
    do {                                                                                   \
        cudaError_t err_ = (expr);                                                         \
        if (err_ != cudaSuccess)                                                           \
            return fail(err_ == cudaErrorMemoryAllocation ? QIEO_ERR_OOM : QIEO_ERR_CUDA, \
                        "%s: %s (%s:%d)", #expr, cudaGetErrorString(err_), __FILE__,       \
                        __LINE__);                                                         \
    } while (0)

constexpr int32_t kMaxD = 4 * qieo::kMaxK;
constexpr double kWaitSeconds = 600.0;
constexpr uint64_t kDefaultBarrierWaitNs = 10ull * 1000 * 1000 * 1000;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int pow2_ceil(int x)
{
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

}  // namespace

namespace qieo_internal {
// Lets the library's other translation units report through qieo_last_error().
void set_last_error(const char *msg) { g_last_error = msg; }
}  // namespace qieo_internal

namespace {

// Launch shapes chosen by qieo_autotune, keyed by (ng, np, D, rule, narrow items).
struct TuneKey {
    int32_t ng, np, D, rule, narrow;
    bool operator<(const TuneKey &o) const
    {
        return std::tie(ng, np, D, rule, narrow) < std::tie(o.ng, o.np, o.D, o.rule, o.narrow);
    }
};
std::mutex g_tune_mutex;
std::map<TuneKey, std::pair<int32_t, int32_t>> g_tuned;   // -> (lanes, warps)

}  // namespace

struct qieo_instance {
    int32_t np = 0, ng = 0, svec = 0, xstride = 0, K = 0, D = 0;
    int32_t rule = 0, host_de = 0, flags = 0;
    int64_t capacity = 0, lambda = 1;
    uint32_t seed = 0, inst_id = 0;
    int device = 0, sm_count = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;

    // problem bounds that decide the sum and elite-key modes
    bool narrow_items = false;     // 0 <= w, v <= 255
    bool state8 = false;           // angle indices stored as bytes (QIEO_FLAG_STATE_I8)
    int64_t sum_w = 0, sum_v = 0, sum_absv = 0;
    bool key_ok = false;

    // device memory (owned unless it was placed in a server's arena)
    void *block = nullptr;
    bool owns_block = true;
    bool fixed_history = false;     // history lives inside an arena block of fixed capacity
    qieo::GenParams gp{};
    const uint4 *items_narrow = nullptr;
    int4 *segq = nullptr;            // segment queue of the deferred forms (own allocation)
    int32_t segq_cap = 0;
    bool seg_delta = false;          // generation kernel forms the R1 deltas once per segment
    int32_t *hist_e = nullptr;
    int64_t *hist_f = nullptr;
    unsigned long long *hist_d = nullptr;   // vectors that did not draw, per generation (in
                                            // hist_f's block)
    int32_t hist_cap = 0;

    // host mirror of the generation counter (number of generations run since reset)
    int32_t t = 0;

    // launch shape
    int32_t lanes = 32, warps = 8, grid = 1, grid_override = 0, narrow = 0;
    size_t smem = 0;
    bool coop = false;             // the run fits one cooperative launch
    bool resident_fits = false;    // each block's share of the state fits in shared memory
    size_t res_smem = 0;           // dynamic shared memory of the resident form
    int32_t res_share = 0;         // tile-rows of the largest share

    // sixteen genes per thread and pass (QIEO_FLAG_SIXTEEN): the geometry of
    // generation_kernel2 (tiles of 512 vectors), its grid, shared memory and segment queue;
    // a launch takes gp and replaces these fields
    bool sixteen = false;
    int32_t max_item = 0;          // largest weight or value
    int32_t ntile2 = 0, seg_rows_max2 = 0, nsegs2 = 0;
    int64_t units2 = 0;
    const int4 *segq2_view = nullptr;
    int32_t grid2 = 0;
    size_t smem2 = 0;
    int4 *segq2 = nullptr;
    int32_t segq2_cap = 0;

    // CUDA graphs keyed by the number of generations of a run; a graph is captured the
    // second time a run length is seen (a one-off run is cheaper to launch directly)
    std::map<int32_t, cudaGraphExec_t> graphs;
    std::map<int32_t, int32_t> run_lengths_seen;

    // kernel timing
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    double kernel_ms = 0.0;
    int64_t kernel_launches = 0;

    // host DetermineElite
    int64_t *h_fit = nullptr;

    // per-step timing (QIEO_FLAG_UNFUSED / elite_on_host with QIEO_FLAG_TIME_KERNELS)
    std::vector<cudaEvent_t> phase_ev;
    double phase_ms[4] = {0.0, 0.0, 0.0, 0.0};
    int64_t phase_gens = 0;

    // per-generation timing (QIEO_FLAG_TIME_GENERATIONS): gen_ev[i] is recorded before the
    // launch of the last run's generation i, gen_ev[gen_ev_n] after its last launch
    std::vector<cudaEvent_t> gen_ev;
    int32_t gen_ev_n = 0;
    // ... or, for a resident-form run, the device clock at each generation's start
    unsigned long long *gen_ns = nullptr;
    int32_t gen_ns_cap = 0;
    bool gen_ns_last = false;

    // a row block of a population sharded by rows (qieo_create_row_block): its rows are
    // chromosomes row0 .. row0 + np - 1 of the whole population; ext_elite holds the
    // packed elite row passed to qieo_rows_rotate; rows_t is the generation last observed
    bool row_block = false;
    uint8_t *ext_elite = nullptr;
    int32_t rows_t = -1;

    // fixed-vector words (qieo_launch_shape.fixed_words): one allocation holding the three
    // per-generation counters (first 256 bytes) and the words; fword_bytes = 0 when the
    // instance keeps none
    void *fword_mem = nullptr;
    size_t fword_bytes = 0;
    size_t fword_state_bytes = 0;      // the counters, words and row totals (cleared together);
                                       // the tile sums after them stay
    bool fword_dirty = false;          // a run since the last clear may have written words
    std::vector<uint32_t> tile_sums;   // per tile of 256 vectors: sum of weights, of values
};

namespace {

void drop_graphs(qieo_instance *q)
{
    for (auto &kv : q->graphs) cudaGraphExecDestroy(kv.second);
    q->graphs.clear();
}

// Kernel instantiation for (narrow sums, rotation rule, asynchronous-copy ring).
template <template <bool, int, bool> class Pick>
typename Pick<true, 0, true>::type kernel_of(const qieo_instance *q, bool ring)
{
    if (q->narrow) {
        if (q->rule) return ring ? Pick<true, 1, true>::get() : Pick<true, 1, false>::get();
        return ring ? Pick<true, 0, true>::get() : Pick<true, 0, false>::get();
    }
    if (q->rule) return ring ? Pick<false, 1, true>::get() : Pick<false, 1, false>::get();
    return ring ? Pick<false, 0, true>::get() : Pick<false, 0, false>::get();
}

template <bool N, int R, bool T>
struct PickGen {
    typedef void (*type)(qieo::GenParams);
    static type get() { return &qieo::generation_kernel<N, R, T>; }
};

template <bool N, int R, bool T>
struct PickRun {
    typedef void (*type)(qieo::GenParams, int32_t);
    static type get() { return &qieo::run_kernel<N, R, T>; }
};

// The generation kernel of an instance (byte-state instances: narrow sums, ring form). With
// seg_delta (rule R1, ring form, segment queue) the variant that forms the CIP deltas once
// per segment.
PickGen<true, 0, true>::type gen_fn(const qieo_instance *q, bool ring, bool seg_delta)
{
    if (q->gp.fword && ring)   // fixed-vector words (R2 forms its rotation per vector)
        return q->rule ? &qieo::generation_kernel<true, 1, true, false, false, true>
                       : &qieo::generation_kernel<true, 0, true, false, true, true>;
    if (seg_delta && ring && q->rule == 0) {
        if (q->state8) return &qieo::generation_kernel<true, 0, true, true, true>;
        return q->narrow ? &qieo::generation_kernel<true, 0, true, false, true>
                         : &qieo::generation_kernel<false, 0, true, false, true>;
    }
    if (q->state8)
        return q->rule ? &qieo::generation_kernel<true, 1, true, true> : &qieo::generation_kernel<true, 0, true, true>;
    return kernel_of<PickGen>(q, ring);
}

PickGen<true, 0, true>::type gen_fn(const qieo_instance *q, bool ring)
{
    return gen_fn(q, ring, q->seg_delta);
}

const void *gen_kernel_of(const qieo_instance *q, bool ring, bool seg_delta)
{
    return reinterpret_cast<const void *>(gen_fn(q, ring, seg_delta));
}

const void *run_kernel_of(const qieo_instance *q, bool ring)
{
    return reinterpret_cast<const void *>(kernel_of<PickRun>(q, ring));
}

// The resident-form run kernel (rule R1 forms its CIP deltas once per segment).
typedef void (*ResidentFn)(qieo::GenParams, int32_t, int32_t);
ResidentFn resident_fn(const qieo_instance *q)
{
    if (q->narrow) return q->rule ? &qieo::resident_run_kernel<true, 1, false> : &qieo::resident_run_kernel<true, 0, true>;
    return q->rule ? &qieo::resident_run_kernel<false, 1, false> : &qieo::resident_run_kernel<false, 0, true>;
}

// Lets the device's default memory pool keep up to 1 GiB of released blocks, so that
// creating and destroying instances in a loop reuses memory instead of mapping it anew
// (set once per device).
void keep_pool_memory(int device)
{
    static std::mutex mu;
    static std::vector<int> done;
    std::lock_guard<std::mutex> lock(mu);
    if (std::find(done.begin(), done.end(), device) != done.end()) return;
    cudaMemPool_t pool = nullptr;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t keep = (uint64_t)1 << 30;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    done.push_back(device);
}

// A pinned host buffer of at least `bytes` for small device-to-host reads, one per host
// thread, grown on demand (pinned memory makes the copies asynchronous, so a read waits
// once).
qieo_status pinned_scratch(size_t bytes, char **out)
{
    struct Scratch {
        char *p = nullptr;
        size_t n = 0;
        ~Scratch()
        {
            if (p) cudaFreeHost(p);
        }
    };
    thread_local Scratch s;
    if (s.n < bytes) {
        if (s.p) cudaFreeHost(s.p);
        s.p = nullptr;
        s.n = 0;
        const size_t n = std::max<size_t>(bytes, 4096);
        CUDA_TRY(cudaMallocHost(&s.p, n));
        s.n = n;
    }
    *out = s.p;
    return QIEO_OK;
}

// The two timing events, made on first use.
qieo_status ensure_events(qieo_instance *q)
{
    if (!q->ev0) CUDA_TRY(cudaEventCreate(&q->ev0));
    if (!q->ev1) CUDA_TRY(cudaEventCreate(&q->ev1));
    return QIEO_OK;
}

// Resident blocks per SM of a kernel at a dynamic shared-memory size (after raising the
// kernel's shared-memory limit to it), cached per (device, kernel, size): instances of the
// same kind then configure without querying the runtime again.
qieo_status resident_blocks(int device, const void *fn, size_t smem, int *bps)
{
    struct Key {
        int device;
        const void *fn;
        size_t smem;
        bool operator<(const Key &o) const { return std::tie(device, fn, smem) < std::tie(o.device, o.fn, o.smem); }
    };
    static std::mutex mu;
    static std::map<Key, int> cache;
    const Key key{device, fn, smem};
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            *bps = it->second;
            return QIEO_OK;
        }
    }
    // The limit is a property of the kernel, shared by every instance that launches it: it
    // is only ever raised (to the largest size asked for on the device), never lowered below
    // what another instance launches with.
    static std::map<std::pair<int, const void *>, size_t> limit;
    std::lock_guard<std::mutex> lock(mu);
    size_t &lim = limit[{device, fn}];
    if (smem > lim) {
        CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        lim = smem;
    }
    int n = 0;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, qieo::kThreads, smem));
    cache[key] = n;
    *bps = n;
    return QIEO_OK;
}

// Segment queue of the deferred forms: the units (tile-rows) in order, cut into segments
// within one tile of at most seg_max rows whose size follows the remaining work (guided
// self-scheduling: remaining / (2 grid), at least kQueueMinRows), so that the first
// segments are large and the last ones small. Only when a block's equal share is at least
// kQueueMinShare tile-rows: with smaller shares the latency each extra segment adds (the
// queue's atomic, the segment's first copies, its flush) costs more than the balance
// gains (measured: 1,024 x 10,000 genes, 8 rows per block, 10.1 -> 12.2 us per generation
// with a queue; 4,096 x 100,000, 330 rows per block, 396 -> 367 us). Instances placed in
// a server arena run in batches only and keep none.
//
// Instances that keep fixed-vector words always take the queue (their generation kernel
// has no other form) and cut it at multiples of 8 rows (f_align; seg_max is then a
// multiple of 8), so that every segment starts on a group of F words.
constexpr int64_t kQueueMinRows = 4;
constexpr int64_t kQueueMinShare = 64;

qieo_status build_queue_into(qieo_instance *q, int64_t units, int grid, int seg_max, bool use_ring, int4 *&buf,
                             int32_t &cap, const int4 *&segq_out, int32_t &nsegs_out, bool f_align = false)
{
    segq_out = nullptr;
    nsegs_out = 0;
    if (!use_ring || !q->owns_block || (!f_align && units < kQueueMinShare * (int64_t)grid)) return QIEO_OK;
    std::vector<int4> segs;
    for (int64_t u = 0; u < units;) {
        const int64_t tile = u / q->np, ra = u - tile * q->np;
        const int64_t rem = units - u;
        int64_t rows = std::max<int64_t>(kQueueMinRows, (rem + 2 * (int64_t)grid - 1) / (2 * (int64_t)grid));
        if (f_align) rows = (rows + 7) / 8 * 8;
        rows = std::min<int64_t>(rows, std::min<int64_t>((int64_t)seg_max, (int64_t)q->np - ra));
        segs.push_back(make_int4((int)tile, (int)ra, (int)rows, 0));
        u += rows;
    }
    if ((int64_t)segs.size() > cap) {
        if (buf) cudaFreeAsync(buf, q->stream);
        buf = nullptr;
        cap = 0;
        keep_pool_memory(q->device);
        CUDA_TRY(cudaMallocAsync(&buf, segs.size() * sizeof(int4), q->stream));
        cap = (int32_t)segs.size();
    }
    CUDA_TRY(cudaMemcpyAsync(buf, segs.data(), segs.size() * sizeof(int4), cudaMemcpyHostToDevice, q->stream));
    segq_out = buf;
    nsegs_out = (int32_t)segs.size();
    return QIEO_OK;
}

qieo_status build_segment_queue(qieo_instance *q, int64_t units, int grid, int seg_max, bool use_ring,
                                bool f_align = false)
{
    return build_queue_into(q, units, grid, seg_max, use_ring, q->segq, q->segq_cap, q->gp.segq, q->gp.nsegs,
                            f_align);
}

// Persistent blocks per SM of the single-instance kernels. The schedulers favour older
// warps, so blocks sharing an SM do not progress equally; measured on the GB300 (per
// 25-generation timing, c2 = 1,024 x 10,000 genes with equal static shares, c3 = 4,096 x
// 100,000 with the segment queue): 4 blocks 10.06 / 366 us per generation, 3 blocks 9.61 /
// 364 us (per-pass deltas), 2 blocks worse (10.7 / 387 us with per-segment deltas).
constexpr int kBlocksPerSm = 3;

// Most dynamic shared memory a block of the resident form may take (of the 227 KB a block
// can have; the kernel's static tables take the rest).
constexpr size_t kResidentMaxSmem = 200 * 1024;

qieo_status configure_sixteen(qieo_instance *q);
bool use_resident(const qieo_instance *q);
bool use_cooperative(const qieo_instance *q);

// Fixed-vector words: kept from the generation after the first whose estimate of fixed
// vectors reaches kFwordOnFraction of the population's vectors; a generation takes the
// sparse form once at least kSparseMinFraction were fixed after the one before.
constexpr double kFwordOnFraction = 0.40;
constexpr double kSparseMinFraction = 0.50;
constexpr int kFwordMaxSegRows = 256;      // a row of a segment fits 8 bits of a list entry

// Whether the instance keeps fixed-vector words: the runs that take the one-launch-per-
// generation deferred form with the generation kernel that maintains them.
bool wants_fword(const qieo_instance *q, bool use_ring)
{
    return !(q->flags & (QIEO_FLAG_NO_FIXED_WORDS | QIEO_FLAG_SIXTEEN | QIEO_FLAG_CONVERGE | QIEO_FLAG_UNFUSED |
                         QIEO_FLAG_COOPERATIVE)) &&
           use_ring && q->narrow && !q->state8 && q->key_ok && !q->host_de && q->lanes == 32 &&
           q->sum_w < ((int64_t)1 << 25) && q->sum_v < ((int64_t)1 << 25) && !q->tile_sums.empty() &&
           q->warps == 8 && q->owns_block && !q->row_block && !use_resident(q) && !use_cooperative(q);
}

// Allocates (all words 0: no vector known to be fixed) or releases the words and fills the
// fields of gp. Words kept from an earlier call of the same geometry stay valid.
qieo_status configure_fword(qieo_instance *q, bool want, int ntile)
{
    qieo::GenParams &g = q->gp;
    // [counters: 256 B][the words: np x fstride bits][row totals: np x 8 B][tile item sums]
    const int32_t fstride = ntile * qieo::kThreads;
    const size_t words = align_up((size_t)q->np * (size_t)(fstride / 32) * sizeof(uint32_t), 256);
    const size_t prev = align_up((size_t)q->np * 8, 256);
    const size_t bytes = want ? 256 + words + prev + (size_t)ntile * 8 : 0;
    if (bytes != q->fword_bytes) {
        if (q->fword_mem) cudaFreeAsync(q->fword_mem, q->stream);
        q->fword_mem = nullptr;
        q->fword_bytes = 0;
        q->fword_state_bytes = 0;
        if (bytes) {
            keep_pool_memory(q->device);
            cudaError_t ce = cudaMallocAsync(&q->fword_mem, bytes, q->stream);
            if (ce != cudaSuccess) {
                g.fword = nullptr;
                g.fcnt = nullptr;
                return fail(ce == cudaErrorMemoryAllocation ? QIEO_ERR_OOM : QIEO_ERR_CUDA,
                            "fixed-vector words (%zu bytes): %s", bytes, cudaGetErrorString(ce));
            }
            q->fword_bytes = bytes;
            q->fword_state_bytes = 256 + words + prev;
            q->fword_dirty = false;
            CUDA_TRY(cudaMemsetAsync(q->fword_mem, 0, bytes, q->stream));
            if ((int)q->tile_sums.size() != 2 * ntile) return fail(QIEO_ERR_INVALID, "internal: tile sums");
            CUDA_TRY(cudaMemcpyAsync(static_cast<char *>(q->fword_mem) + 256 + words + prev, q->tile_sums.data(),
                                     (size_t)ntile * 8, cudaMemcpyHostToDevice, q->stream));
        }
    }
    char *base = static_cast<char *>(q->fword_mem);
    g.fcnt = bytes ? reinterpret_cast<unsigned long long *>(base) : nullptr;
    g.fword = bytes ? reinterpret_cast<uint32_t *>(base + 256) : nullptr;
    g.fprev = bytes ? reinterpret_cast<unsigned long long *>(base + 256 + words) : nullptr;
    g.ftile = bytes ? reinterpret_cast<const uint32_t *>(base + 256 + words + prev) : nullptr;
    g.fsum_w = q->sum_w;
    g.fsum_v = q->sum_v;
    g.fstride = fstride;
    const double vecs = (double)q->np * (double)q->svec;
    const double need = std::ceil(kSparseMinFraction * vecs), on = std::ceil(kFwordOnFraction * vecs);
    const bool always = (q->flags & QIEO_FLAG_SPARSE_ALWAYS) != 0;
    g.sparse_min = always ? 0ull : (unsigned long long)need;
    g.f_on_min = always ? 0ull : (unsigned long long)on;
    return QIEO_OK;
}

// Every fixed-vector word to 0 (after the state changed outside the kernels that keep them),
// with the counters and row totals; the tile sums stay. Nothing to do when no run of the
// kernel that keeps them has happened since the words were last cleared (a batch member that
// only runs in batches).
qieo_status clear_fword(qieo_instance *q, cudaStream_t s)
{
    if (q->fword_state_bytes && q->fword_dirty) CUDA_TRY(cudaMemsetAsync(q->fword_mem, 0, q->fword_state_bytes, s));
    q->fword_dirty = false;
    return QIEO_OK;
}

// Picks the sum mode and the persistent grid for the current tile (lanes x warps) and
// fills the launch fields of gp.
qieo_status configure(qieo_instance *q)
{
    const int tile = q->lanes * q->warps;
    const int rpp = qieo::kThreads / tile;
    const int ntile = (q->svec + tile - 1) / tile;
    // 16-bit packed sums inside a warp need items <= 255 (256 genes * 255 < 2^16); the
    // packed row word (count << 52 | SV << 26 | SW) needs row sums < 2^26 and at most 4095
    // tiles per row.
    q->narrow = (!(q->flags & QIEO_FLAG_FORCE_WIDE) && q->narrow_items &&
                 q->sum_w < (1ll << 26) && q->sum_v < (1ll << 26) && ntile <= 4095) ? 1 : 0;
    const int64_t units = (int64_t)ntile * q->np;
    const size_t row_bytes = q->narrow ? 8 : 16;
    if (q->state8 && !q->narrow)
        return fail(QIEO_ERR_INVALID, "QIEO_FLAG_STATE_I8 needs the packed item sums: items in [0, 255], "
                    "item sums below 2^26 and at most 4095 tiles per row");

    // The state streams through the per-thread cp.async ring unless register prefetch is
    // asked for.
    const bool use_ring = !(q->flags & QIEO_FLAG_REGISTER_PREFETCH);
    const size_t ring = use_ring ? qieo::kRingBytes : 0;

    // Blocks resident at once, for the larger of the shared-memory sizes used and either
    // generation-kernel variant, capped at kBlocksPerSm.
    const size_t smem0 = ring + (size_t)qieo::kMaxSegRows * row_bytes;
    int bps_gen = 0, bps_sd = 0, bps_run = 0, bps_f = kBlocksPerSm;
    qieo_status ost = resident_blocks(q->device, gen_kernel_of(q, use_ring, false), smem0, &bps_gen);
    if (ost == QIEO_OK) ost = resident_blocks(q->device, gen_kernel_of(q, use_ring, true), smem0, &bps_sd);
    if (ost == QIEO_OK) ost = resident_blocks(q->device, run_kernel_of(q, use_ring), smem0, &bps_run);
    if (ost == QIEO_OK && use_ring && q->narrow && !q->state8)
        ost = resident_blocks(q->device,
                              q->rule ? reinterpret_cast<const void *>(&qieo::generation_kernel<true, 1, true, false, false, true>)
                                      : reinterpret_cast<const void *>(&qieo::generation_kernel<true, 0, true, false, true, true>),
                              ring + (size_t)kFwordMaxSegRows * row_bytes, &bps_f);
    if (ost != QIEO_OK) return ost;
    const int bps = std::min(std::min(kBlocksPerSm, bps_f), std::min(bps_gen, std::min(bps_sd, bps_run)));
    const int64_t resident = (int64_t)q->sm_count * std::max(1, bps);
    int grid = q->grid_override;
    if (grid <= 0) {
        const int64_t by_work = (units + rpp - 1) / rpp;
        grid = (int)std::max<int64_t>(1, std::min<int64_t>(resident, by_work));
    }
    const int64_t share = (units + grid - 1) / grid;
    int seg_max = (int)std::max<int64_t>(1, std::min<int64_t>(qieo::kMaxSegRows, share));
    q->grid = grid;
    q->smem = ring + (size_t)seg_max * row_bytes;
    q->coop = bps_run > 0 && grid <= (int64_t)q->sm_count * bps_run;
    q->gp.ring = use_ring ? 1 : 0;

    // Resident form: every block's share of the state (share tile-rows x tile vectors of
    // 16 bytes) stays in its shared memory for a whole run; possible when all blocks of
    // the grid fit on the device at once with that much shared memory each.
    q->resident_fits = false;
    q->res_share = (int32_t)share;
    q->res_smem = (size_t)share * tile * sizeof(uint4) + (size_t)seg_max * row_bytes;
    if (q->res_smem <= kResidentMaxSmem && !q->state8) {
        int bps_res = 0;
        qieo_status rst = resident_blocks(q->device, reinterpret_cast<const void *>(resident_fn(q)),
                                          q->res_smem, &bps_res);
        if (rst != QIEO_OK) return rst;
        q->resident_fits = bps_res > 0 && grid <= (int64_t)q->sm_count * bps_res;
    }

    // fixed-vector words: segments of at most 256 rows, cut at multiples of 8
    const bool want_f = wants_fword(q, use_ring);
    if (want_f) {
        seg_max = std::min(kFwordMaxSegRows, std::max(8, seg_max & ~7));
        q->smem = ring + (size_t)seg_max * row_bytes;
    }

    qieo::GenParams &g = q->gp;
    g.items_narrow = q->items_narrow;
    g.ntile = ntile;
    g.units = units;
    g.lanes = q->lanes;
    g.warps = q->warps;
    g.seg_rows_max = seg_max;
    g.key_mode = q->key_ok ? 1 : 0;
    qieo_status qst = build_segment_queue(q, units, grid, seg_max, use_ring, want_f);
    if (qst != QIEO_OK) return qst;
    qst = configure_fword(q, want_f && g.nsegs > 0, ntile);
    if (qst != QIEO_OK) return qst;
    q->seg_delta = g.nsegs > 0 && q->rule == 0;   // long queued segments: deltas per segment
    drop_graphs(q);
    return configure_sixteen(q);
}

void default_tile(qieo_instance *q)
{
    const int svec = q->svec;
    if (svec <= 16) {
        q->lanes = pow2_ceil(svec);
        q->warps = 1;
    } else {
        q->lanes = 32;
        q->warps = std::min(8, pow2_ceil((svec + 31) / 32));
    }
}

cudaLaunchConfig_t launch_config(const qieo_instance *q, dim3 grid, size_t smem,
                                 cudaLaunchAttribute *attr)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(qieo::kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = q->stream;
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

// One generation launch. deferred_g >= 0 selects the deferred close (generation *gen +
// deferred_g of the run); -1 the close by the last block (the generation counter advances
// per launch).
cudaError_t launch_gen(const qieo_instance *q, int apply_cip, int do_de, int32_t deferred_g = -1)
{
    if (q->sixteen && deferred_g >= 0) {   // 16 genes per thread and pass (deferred close)
        qieo::GenParams p = q->gp;
        p.ntile = q->ntile2;
        p.units = q->units2;
        p.seg_rows_max = q->seg_rows_max2;
        p.segq = q->segq2_view;
        p.nsegs = q->nsegs2;
        p.apply_cip = apply_cip;
        p.do_de = do_de;
        p.deferred = 1;
        p.g = deferred_g;
        cudaLaunchAttribute attr[1];
        cudaLaunchConfig_t cfg = launch_config(q, dim3(q->grid2), q->smem2, attr);
        return cudaLaunchKernelEx(&cfg, qieo::generation_kernel2, p);
    }
    qieo::GenParams p = q->gp;
    p.apply_cip = apply_cip;
    p.do_de = do_de;
    p.deferred = deferred_g >= 0 ? 1 : 0;
    p.g = deferred_g >= 0 ? deferred_g : 0;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = launch_config(q, dim3(q->grid), q->smem, attr);
    return cudaLaunchKernelEx(&cfg, gen_fn(q, q->gp.ring != 0), p);
}

// One cooperative launch for a run of G generations. With the packed elite key the run uses
// the deferred close (a plain grid barrier between generations) and a one-thread launch
// then advances the generation counter; otherwise the last block closes each generation.
cudaError_t launch_run(const qieo_instance *q, int32_t G)
{
    qieo::GenParams p = q->gp;
    p.deferred = q->key_ok ? 1 : 0;
    p.g = 0;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(q->grid);
    cfg.blockDim = dim3(qieo::kThreads);
    cfg.dynamicSmemBytes = q->smem;
    cfg.stream = q->stream;
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t ce = cudaLaunchKernelEx(&cfg, kernel_of<PickRun>(q, q->gp.ring != 0), p, G);
    if (ce != cudaSuccess || !p.deferred) return ce;
    cudaLaunchAttribute attr1[1];
    cudaLaunchConfig_t one = launch_config(q, dim3(1), 0, attr1);
    one.blockDim = dim3(32);
    return cudaLaunchKernelEx(&one, qieo::end_run_kernel, p, G);
}

cudaError_t launch_final_cip(const qieo_instance *q, int32_t deferred_G = 0)
{
    const size_t total = (size_t)q->np * q->svec;
    const int blocks = (int)std::max<size_t>(
        1, std::min<size_t>((total + qieo::kThreads - 1) / qieo::kThreads,
                            (size_t)std::max(q->sm_count, 1) * 8));
    qieo::GenParams p = q->gp;
    p.deferred = deferred_G > 0 ? 1 : 0;
    p.g = deferred_G;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = launch_config(q, dim3(blocks), 0, attr);
    cudaError_t ce = q->rule ? cudaLaunchKernelEx(&cfg, qieo::cip_kernel<1>, p)
                             : cudaLaunchKernelEx(&cfg, qieo::cip_kernel<0>, p);
    if (ce != cudaSuccess || deferred_G <= 0) return ce;
    cudaLaunchConfig_t one = launch_config(q, dim3(1), 0, attr);
    one.blockDim = dim3(32);
    return cudaLaunchKernelEx(&one, qieo::end_run_kernel, p, deferred_G);
}

qieo_status wait_stream(cudaStream_t s)
{
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t e = cudaStreamQuery(s);
        if (e == cudaSuccess) return QIEO_OK;
        if (e != cudaErrorNotReady)
            return fail(QIEO_ERR_CUDA, "device work failed: %s", cudaGetErrorString(e));
        const double el =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > kWaitSeconds)
            return fail(QIEO_ERR_TIMEOUT, "device work did not finish within %.0f s", kWaitSeconds);
        // poll without sleeping for the first 200 us (a sleep is at least tens of us on
        // Linux, longer than most short waits), then back off
        if (el < 2e-4) std::this_thread::yield();
        else std::this_thread::sleep_for(std::chrono::microseconds(el < 0.01 ? 20 : 200));
    }
}

// Threshold table T[n] = round(sin^2(n pi / D) 2^32), evaluated as 2^31 (1 - cos(2 n pi/D))
// in extended precision for n <= K and mirrored (T[2K-n] = 2^32 - T[n]) above.
void build_thresholds(int32_t D, std::vector<uint64_t> &T)
{
    const int32_t K = D / 4;
    T.assign((size_t)(2 * K + 1), 0);
    const long double pi = acosl(-1.0L);
    for (int32_t n = 0; n <= K; ++n) {
        const long double c = cosl(2.0L * pi * (long double)n / (long double)D);
        const long double val = 2147483648.0L * (1.0L - c);
        T[(size_t)n] = (uint64_t)llroundl(val);
    }
    T[0] = 0;
    T[(size_t)K] = 1ull << 31;
    for (int32_t n = K + 1; n <= 2 * K; ++n) T[(size_t)n] = (1ull << 32) - T[(size_t)(2 * K - n)];
}

}  // namespace

namespace qieo_internal {
// The threshold table for the library's other translation units.
void build_thresholds(int32_t D, std::vector<uint64_t> &T) { ::build_thresholds(D, T); }
}  // namespace qieo_internal

namespace {

qieo_status ensure_history(qieo_instance *q, int32_t need)
{
    if (need <= q->hist_cap) return QIEO_OK;
    if (q->fixed_history)
        return fail(QIEO_ERR_INVALID, "generation %d beyond the %d generations reserved for this solve",
                    need, q->hist_cap);
    int32_t cap = std::max<int32_t>(need, std::max<int32_t>(1024, q->hist_cap * 2));
    int32_t *e = nullptr;
    int64_t *f = nullptr;
    keep_pool_memory(q->device);
    CUDA_TRY(cudaMallocAsync(&e, (size_t)cap * sizeof(int32_t), q->stream));
    // the fitness history, then the counts of vectors that did not draw
    // (qieo_get_drawn_vectors)
    cudaError_t err = cudaMallocAsync(&f, (size_t)cap * 2 * sizeof(int64_t), q->stream);
    if (err != cudaSuccess) {
        cudaFreeAsync(e, q->stream);
        return fail(QIEO_ERR_OOM, "history buffer: %s", cudaGetErrorString(err));
    }
    unsigned long long *d = reinterpret_cast<unsigned long long *>(f + cap);
    CUDA_TRY(cudaMemsetAsync(d, 0, (size_t)cap * sizeof(unsigned long long), q->stream));
    if (q->hist_cap > 0) {
        CUDA_TRY(cudaMemcpyAsync(e, q->hist_e, (size_t)q->hist_cap * sizeof(int32_t),
                                 cudaMemcpyDeviceToDevice, q->stream));
        CUDA_TRY(cudaMemcpyAsync(f, q->hist_f, (size_t)q->hist_cap * sizeof(int64_t),
                                 cudaMemcpyDeviceToDevice, q->stream));
        CUDA_TRY(cudaMemcpyAsync(d, q->hist_d, (size_t)q->hist_cap * sizeof(unsigned long long),
                                 cudaMemcpyDeviceToDevice, q->stream));
        cudaFreeAsync(q->hist_e, q->stream);
        cudaFreeAsync(q->hist_f, q->stream);
    }
    q->hist_e = e;
    q->hist_f = f;
    q->hist_d = d;
    q->hist_cap = cap;
    q->gp.hist_e = e;
    q->gp.hist_f = f;
    q->gp.hist_d = d;
    drop_graphs(q);
    return QIEO_OK;
}

qieo_status enqueue_device_run(qieo_instance *q, int32_t G)
{
    if (q->flags & QIEO_FLAG_TIME_KERNELS) CUDA_TRY(cudaEventRecord(q->ev0, q->stream));
    // Deferred close whenever the elite key holds the fitness (the generation counter then
    // advances once per run); otherwise the last block of each generation closes it.
    const bool deferred = q->key_ok;
    const bool per_gen = (q->flags & QIEO_FLAG_TIME_GENERATIONS) != 0;
    if (per_gen) {
        while (q->gen_ev.size() < (size_t)G + 1) {
            cudaEvent_t e = nullptr;
            CUDA_TRY(cudaEventCreate(&e));
            q->gen_ev.push_back(e);
        }
        q->gen_ev_n = 0;
        q->gen_ns_last = false;
    }
    for (int32_t g = 0; g < G; ++g) {
        if (per_gen) CUDA_TRY(cudaEventRecord(q->gen_ev[(size_t)g], q->stream));
        CUDA_TRY(launch_gen(q, g > 0 ? 1 : 0, 1, deferred ? g : -1));
    }
    if (per_gen) {
        CUDA_TRY(cudaEventRecord(q->gen_ev[(size_t)G], q->stream));
        q->gen_ev_n = G;
    }
    if (q->flags & QIEO_FLAG_TIME_KERNELS) CUDA_TRY(cudaEventRecord(q->ev1, q->stream));
    CUDA_TRY(launch_final_cip(q, deferred ? G : 0));
    return QIEO_OK;
}

// A run as one cooperative launch: when asked for, or by default for small instances
// (at most 2^22 genes) with the packed elite key, where the grid barrier costs less than a
// launch per generation (measured: 64 x 100 genes 2.86 vs 3.44 us per generation; at
// 1,024 x 10,000 the two are within 1 %, at 4,096 x 100,000 the cooperative form is 2 %
// slower). Not with the convergence test or byte state.
// The resident form (see resident_run_kernel) is used whenever it fits, unless a flag asks
// for one launch per generation, the streamed form or the cooperative streamed form.
bool use_resident(const qieo_instance *q)
{
    if (!q->resident_fits || q->host_de || q->row_block || !q->key_ok || q->state8) return false;
    return !(q->flags & (QIEO_FLAG_UNFUSED | QIEO_FLAG_PER_GENERATION | QIEO_FLAG_CONVERGE |
                         QIEO_FLAG_COOPERATIVE | QIEO_FLAG_STREAMED));
}

bool use_cooperative(const qieo_instance *q);

// Sixteen genes per thread and pass (generation_kernel2), when asked for and the run takes
// the deferred one-launch-per-generation form: rule R1, packed items of at most 127, 16-bit
// state, the default tile (32 lanes x 8 warps), no convergence test. Its tiles are 512
// vectors; gp2 carries their geometry and segment queue, gp keeps the 8-gene one for every
// other launch (batches, cooperative and resident forms, the final CIP).
qieo_status configure_sixteen(qieo_instance *q)
{
    q->sixteen = false;
    if (!(q->flags & QIEO_FLAG_SIXTEEN) || !q->narrow || q->max_item > 127 || q->rule != 0 || q->state8 ||
        !q->gp.ring || !q->key_ok || q->host_de || (q->flags & (QIEO_FLAG_CONVERGE | QIEO_FLAG_UNFUSED)) ||
        q->lanes != 32 || q->warps != 8 || q->row_block || !q->owns_block || use_resident(q) ||
        use_cooperative(q))
        return QIEO_OK;
    constexpr int kTileVecs = 2 * qieo::kThreads;
    const int ntile = (q->svec + kTileVecs - 1) / kTileVecs;
    if (ntile > 4095) return QIEO_OK;
    const int64_t units = (int64_t)ntile * q->np;
    const size_t ring = (size_t)qieo::kRing2Stages * 2 * qieo::kThreads * sizeof(uint4);
    const size_t smem0 = ring + (size_t)qieo::kMaxSegRows * 8;
    int bps = 0;
    qieo_status st = resident_blocks(q->device, reinterpret_cast<const void *>(qieo::generation_kernel2), smem0, &bps);
    if (st != QIEO_OK) return st;
    if (bps < 1) return QIEO_OK;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)q->sm_count * std::min(bps, 2), units));
    const int64_t share = (units + grid - 1) / grid;
    const int seg_max = (int)std::max<int64_t>(1, std::min<int64_t>(qieo::kMaxSegRows, share));
    q->ntile2 = ntile;
    q->units2 = units;
    q->seg_rows_max2 = seg_max;
    st = build_queue_into(q, units, grid, seg_max, true, q->segq2, q->segq2_cap, q->segq2_view, q->nsegs2);
    if (st != QIEO_OK) return st;
    q->grid2 = grid;
    q->smem2 = ring + (size_t)seg_max * 8;
    q->sixteen = true;
    return QIEO_OK;
}

bool use_cooperative(const qieo_instance *q)
{
    if (!q->coop || q->host_de ||
        (q->flags & (QIEO_FLAG_UNFUSED | QIEO_FLAG_PER_GENERATION | QIEO_FLAG_TIME_GENERATIONS)))
        return false;
    if (q->flags & QIEO_FLAG_COOPERATIVE) return true;
    return q->key_ok && !(q->flags & QIEO_FLAG_CONVERGE) && !q->state8 &&
           (int64_t)q->np * q->svec * 8 <= ((int64_t)1 << 22);
}

// One resident-form run of G generations (one cooperative launch) and the one-thread launch
// that then advances the generation counter.
cudaError_t launch_resident(const qieo_instance *q, int32_t G, unsigned long long *gen_ns)
{
    qieo::GenParams p = q->gp;
    p.deferred = 1;
    p.g = 0;
    p.gen_ns = gen_ns;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(q->grid);
    cfg.blockDim = dim3(qieo::kThreads);
    cfg.dynamicSmemBytes = q->res_smem;
    cfg.stream = q->stream;
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t ce = cudaLaunchKernelEx(&cfg, resident_fn(q), p, G, q->res_share);
    if (ce != cudaSuccess) return ce;
    cudaLaunchAttribute attr1[1];
    cudaLaunchConfig_t one = launch_config(q, dim3(1), 0, attr1);
    one.blockDim = dim3(32);
    return cudaLaunchKernelEx(&one, qieo::end_run_kernel, p, G);
}

qieo_status run_cooperative(qieo_instance *q, int32_t G)
{
    const bool timing = (q->flags & QIEO_FLAG_TIME_KERNELS) != 0;
    const bool resident = use_resident(q);
    if (timing) CUDA_TRY(cudaEventRecord(q->ev0, q->stream));
    // the barrier counts G x grid arrivals in 32 bits: split longer runs (run(a) + run(b)
    // equals run(a + b))
    const int32_t chunk = (int32_t)std::max<int64_t>(1, std::min<int64_t>(G, ((int64_t)1 << 30) / std::max(1, q->grid)));
    const bool stamps = resident && (q->flags & QIEO_FLAG_TIME_GENERATIONS);
    if (stamps && q->gen_ns_cap < G + 1) {
        if (q->gen_ns) cudaFreeAsync(q->gen_ns, q->stream);
        q->gen_ns = nullptr;
        q->gen_ns_cap = 0;
        CUDA_TRY(cudaMallocAsync(&q->gen_ns, (size_t)(G + 1) * sizeof(unsigned long long), q->stream));
        q->gen_ns_cap = G + 1;
    }
    for (int32_t done = 0; done < G; done += chunk)
        CUDA_TRY(resident ? launch_resident(q, std::min(chunk, G - done), stamps ? q->gen_ns + done : nullptr)
                          : launch_run(q, std::min(chunk, G - done)));
    if (stamps) {
        q->gen_ev_n = G;
        q->gen_ns_last = true;
    }
    if (timing) {
        CUDA_TRY(cudaEventRecord(q->ev1, q->stream));
        qieo_status st = wait_stream(q->stream);
        if (st != QIEO_OK) return st;
        float ms = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&ms, q->ev0, q->ev1));
        q->kernel_ms += ms;
        q->kernel_launches += 1;
    }
    return QIEO_OK;
}

qieo_status run_device(qieo_instance *q, int32_t G)
{
    if (q->flags & QIEO_FLAG_TIME_KERNELS) {
        qieo_status st = ensure_events(q);
        if (st != QIEO_OK) return st;
    }
    if (use_resident(q) || use_cooperative(q)) return run_cooperative(q, G);
    if (q->gp.fword) q->fword_dirty = true;
    const bool timing = (q->flags & QIEO_FLAG_TIME_KERNELS) != 0;
    const bool first_time = q->run_lengths_seen[G]++ == 0;
    if ((q->flags & (QIEO_FLAG_NO_GRAPH | QIEO_FLAG_TIME_GENERATIONS)) || (first_time && !q->graphs.count(G))) {
        qieo_status st = enqueue_device_run(q, G);
        if (st != QIEO_OK) return st;
    } else {
        auto it = q->graphs.find(G);
        cudaGraphExec_t exec = nullptr;
        if (it == q->graphs.end()) {
            if (q->graphs.size() >= 8) drop_graphs(q);
            cudaGraph_t graph = nullptr;
            CUDA_TRY(cudaStreamBeginCapture(q->stream, cudaStreamCaptureModeThreadLocal));
            qieo_status st = enqueue_device_run(q, G);
            cudaError_t ce = cudaStreamEndCapture(q->stream, &graph);
            if (st != QIEO_OK) {
                if (graph) cudaGraphDestroy(graph);
                return st;
            }
            if (ce != cudaSuccess) return fail(QIEO_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ce));
            ce = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ce != cudaSuccess) return fail(QIEO_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ce));
            q->graphs[G] = exec;
        } else {
            exec = it->second;
        }
        CUDA_TRY(cudaGraphLaunch(exec, q->stream));
    }
    if (timing && G > 0) {
        qieo_status st = wait_stream(q->stream);
        if (st != QIEO_OK) return st;
        float ms = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&ms, q->ev0, q->ev1));
        q->kernel_ms += ms;
        q->kernel_launches += G;
    }
    return QIEO_OK;
}

qieo_status run_host_de(qieo_instance *q, int32_t G)
{
    const bool timing = (q->flags & QIEO_FLAG_TIME_KERNELS) != 0;
    for (int32_t g = 0; g < G; ++g) {
        CUDA_TRY(launch_gen(q, g > 0 ? 1 : 0, 0));
        std::chrono::steady_clock::time_point t0;
        if (timing) {   // DetermineElite's share starts once the generation kernel is done
            qieo_status st = wait_stream(q->stream);
            if (st != QIEO_OK) return st;
            t0 = std::chrono::steady_clock::now();
        }
        CUDA_TRY(cudaMemcpyAsync(q->h_fit, q->gp.fitness, (size_t)q->np * sizeof(int64_t),
                                 cudaMemcpyDeviceToHost, q->stream));
        qieo_status st = wait_stream(q->stream);
        if (st != QIEO_OK) return st;
        int32_t e = 0;
        for (int32_t c = 1; c < q->np; ++c)
            if (q->h_fit[c] > q->h_fit[e]) e = c;
        qieo::record_elite_kernel<<<1, qieo::kThreads, 0, q->stream>>>(q->gp, e);
        CUDA_TRY(cudaGetLastError());
        if (timing) {
            q->phase_ms[3] += 1e3 * std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            q->phase_gens += 1;
        }
    }
    CUDA_TRY(launch_final_cip(q));
    return wait_stream(q->stream);
}

// The four steps of each generation as four launches (QIEO_FLAG_UNFUSED): CIP toward the
// previous elite (not in a run's first generation: the previous run ended with it), QIP,
// Evaluation, DetermineElite; then the final CIP of the run. With QIEO_FLAG_TIME_KERNELS an
// event is recorded around every launch and the run waits to add up the steps' times.
qieo_status run_unfused(qieo_instance *q, int32_t G)
{
    const bool timing = (q->flags & QIEO_FLAG_TIME_KERNELS) != 0;
    const size_t total = (size_t)q->np * q->svec;
    const int blocks = (int)std::max<size_t>(
        1, std::min<size_t>((total + qieo::kThreads - 1) / qieo::kThreads, (size_t)std::max(q->sm_count, 1) * 8));
    const int eval_blocks = std::max(1, std::min(q->np, std::max(q->sm_count, 1) * 8));
    size_t need = timing ? (size_t)4 * G + 1 : 0;
    while (q->phase_ev.size() < need) {
        cudaEvent_t e = nullptr;
        CUDA_TRY(cudaEventCreate(&e));
        q->phase_ev.push_back(e);
    }
    std::vector<int> phase_of;   // phase of the launch that ends at event i + 1
    size_t ev = 0;
    auto mark = [&](int phase) -> cudaError_t {
        if (!timing) return cudaSuccess;
        if (phase >= 0) phase_of.push_back(phase);
        return cudaEventRecord(q->phase_ev[ev++], q->stream);
    };
    CUDA_TRY(mark(-1));
    for (int32_t g = 0; g < G; ++g) {
        if (g > 0) {
            if (q->rule) qieo::cip_kernel<1><<<blocks, qieo::kThreads, 0, q->stream>>>(q->gp);
            else qieo::cip_kernel<0><<<blocks, qieo::kThreads, 0, q->stream>>>(q->gp);
            CUDA_TRY(cudaGetLastError());
            CUDA_TRY(mark(0));
        }
        qieo::qip_kernel<<<blocks, qieo::kThreads, 0, q->stream>>>(q->gp);
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(mark(1));
        qieo::eval_kernel<<<eval_blocks, qieo::kThreads, 0, q->stream>>>(q->gp);
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(mark(2));
        qieo::de_kernel<<<1, qieo::kThreads, 0, q->stream>>>(q->gp);
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(mark(3));
    }
    CUDA_TRY(launch_final_cip(q));
    if (timing) {
        qieo_status st = wait_stream(q->stream);
        if (st != QIEO_OK) return st;
        for (size_t i = 0; i < phase_of.size(); ++i) {
            float ms = 0.f;
            CUDA_TRY(cudaEventElapsedTime(&ms, q->phase_ev[i], q->phase_ev[i + 1]));
            q->phase_ms[phase_of[i]] += ms;
        }
        q->phase_gens += G;
    }
    return QIEO_OK;
}

// Waits for the instance's stream and reports a device-side wait that ran out.
qieo_status wait_checked(qieo_instance *q)
{
    qieo_status st = wait_stream(q->stream);
    if (st != QIEO_OK) return st;
    int32_t err = 0;
    CUDA_TRY(cudaMemcpyAsync(&err, q->gp.error, sizeof err, cudaMemcpyDeviceToHost, q->stream));
    st = wait_stream(q->stream);
    if (st != QIEO_OK) return st;
    if (err & qieo::kErrBarrierTimeout)
        return fail(QIEO_ERR_TIMEOUT, "a grid-barrier wait inside the run ran out (%.3f s bound); "
                    "the instance state is undefined until qieo_reset", (double)q->gp.wait_ns * 1e-9);
    if (err & qieo::kErrEliteRange)
        return fail(QIEO_ERR_CUDA, "internal error: a generation closed without an elite in "
                    "[0, np); the instance state is undefined until qieo_reset");
    return QIEO_OK;
}

qieo_status check_inst(const qieo_instance *q)
{
    if (!q) return fail(QIEO_ERR_INVALID, "instance is NULL");
    return QIEO_OK;
}

qieo_status set_device(const qieo_instance *q)
{
    CUDA_TRY(cudaSetDevice(q->device));
    return QIEO_OK;
}

}  // namespace

extern "C" {

void qieo_default_params(qieo_params *p)
{
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->np = 64;
    p->dtheta_den = 100;
    p->penalty_lambda = 1;
    p->seed = 1;
    p->instance_id = 0;
    p->rotate_rule = QIEO_RULE_R1;
    p->elite_on_host = 0;
    p->flags = 0;
    p->stream = nullptr;
}

const char *qieo_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

namespace {

// Device memory of one instance, every part 256-byte aligned:
//  0 state | 1 xbits (2 planes) | 2 packed items | 3 wide items | 4 best row | 5 acc |
//  6 cnt | 7 fitness | 8 best[3] | 9 gen | 10 ticket | 11 key | 12 elite idx | 13 thr |
//  14 barrier generation | 15 error word | 16, 17 elite history (only when placed in a
//  server arena with a fixed number of generations)
constexpr int kParts = 18;

size_t instance_layout(int32_t ng, int32_t np, int32_t D, int32_t hist_cap, size_t *off,
                       bool state8 = false)
{
    const size_t svec = (size_t)(ng + 7) / 8;
    const size_t xstride = align_up(svec, 16);
    const size_t ngp = svec * 8;
    const size_t sizes[kParts] = {(size_t)np * svec * (state8 ? sizeof(uint2) : sizeof(uint4)),
                                  2 * (size_t)np * xstride,
                                  ngp * 6,
                                  ngp * 8,
                                  xstride,
                                  (size_t)np * 2 * sizeof(unsigned long long),
                                  (size_t)np * sizeof(unsigned int),
                                  (size_t)np * sizeof(int64_t),
                                  3 * sizeof(int64_t),
                                  sizeof(int32_t),
                                  sizeof(unsigned int),
                                  3 * sizeof(unsigned long long),   // elite key slots
                                  sizeof(int32_t),
                                  (size_t)(D / 2 + 1) * sizeof(uint32_t),
                                  sizeof(int32_t),
                                  8 * sizeof(int32_t),   // error word, convergence words,
                                                         // segment-queue counters
                                  (size_t)hist_cap * sizeof(int32_t),
                                  (size_t)hist_cap * sizeof(int64_t)};
    size_t total = 0;
    for (int i = 0; i < kParts; ++i) {
        off[i] = total;
        total = align_up(total + sizes[i], 256);
    }
    return total;
}

// An instance placed in memory the caller reserved (a server arena).
struct Placement {
    void *block;
    size_t bytes;
    int32_t hist_cap;
};

qieo_status create_instance_impl(const qieo_problem *pr, const qieo_params *pa,
                                 const Placement *ext, bool sync, qieo_instance **out)
{
    if (out) *out = nullptr;
    if (!pr || !pa || !out) return fail(QIEO_ERR_INVALID, "NULL argument");
    if (pr->ng < 1) return fail(QIEO_ERR_INVALID, "ng must be >= 1 (got %d)", pr->ng);
    if (!pr->weights || !pr->values) return fail(QIEO_ERR_INVALID, "weights/values are NULL");
    if (pa->np < 1) return fail(QIEO_ERR_INVALID, "np must be >= 1 (got %d)", pa->np);
    if (pa->dtheta_den < 4 || pa->dtheta_den > kMaxD || pa->dtheta_den % 4 != 0)
        return fail(QIEO_ERR_INVALID, "dtheta_den must be a multiple of 4 in [4, %d] (got %d)",
                    kMaxD, pa->dtheta_den);
    if (pa->penalty_lambda < 1) return fail(QIEO_ERR_INVALID, "penalty_lambda must be >= 1");
    if (pa->rotate_rule != QIEO_RULE_R1 && pa->rotate_rule != QIEO_RULE_R2)
        return fail(QIEO_ERR_INVALID, "rotate_rule must be 0 (R1) or 1 (R2)");
    if (pa->elite_on_host != 0 && pa->elite_on_host != 1)
        return fail(QIEO_ERR_INVALID, "elite_on_host must be 0 or 1");
    if (pr->capacity < 0) return fail(QIEO_ERR_INVALID, "capacity must be >= 0");
    if ((pa->flags & QIEO_FLAG_UNFUSED) && (pa->elite_on_host || (pa->flags & QIEO_FLAG_COOPERATIVE)))
        return fail(QIEO_ERR_INVALID, "QIEO_FLAG_UNFUSED excludes elite_on_host and QIEO_FLAG_COOPERATIVE");
    if ((pa->flags & QIEO_FLAG_STATE_I8) &&
        (pa->dtheta_den > 120 || (pa->flags & (QIEO_FLAG_REGISTER_PREFETCH | QIEO_FLAG_COOPERATIVE |
                                               QIEO_FLAG_UNFUSED | QIEO_FLAG_FORCE_WIDE))))
        return fail(QIEO_ERR_INVALID, "QIEO_FLAG_STATE_I8 needs dtheta_den <= 120 and excludes "
                    "QIEO_FLAG_REGISTER_PREFETCH, QIEO_FLAG_COOPERATIVE, QIEO_FLAG_UNFUSED and "
                    "QIEO_FLAG_FORCE_WIDE");
    if ((pa->flags & QIEO_FLAG_TIME_GENERATIONS) &&
        (pa->elite_on_host || (pa->flags & (QIEO_FLAG_COOPERATIVE | QIEO_FLAG_UNFUSED))))
        return fail(QIEO_ERR_INVALID, "QIEO_FLAG_TIME_GENERATIONS excludes elite_on_host, "
                    "QIEO_FLAG_COOPERATIVE and QIEO_FLAG_UNFUSED");
    if ((pa->flags & QIEO_FLAG_CONVERGE) &&
        (pa->elite_on_host || (pa->flags & (QIEO_FLAG_COOPERATIVE | QIEO_FLAG_UNFUSED))))
        return fail(QIEO_ERR_INVALID, "QIEO_FLAG_CONVERGE excludes elite_on_host, QIEO_FLAG_COOPERATIVE "
                    "and QIEO_FLAG_UNFUSED");

    int64_t sum_w = 0, sum_v = 0, sum_absv = 0;
    int32_t max_w = 0, max_v = 0, min_v = 0;
    for (int32_t j = 0; j < pr->ng; ++j) {
        if (pr->weights[j] < 0) return fail(QIEO_ERR_INVALID, "weight %d is negative", j);
        sum_w += pr->weights[j];
        sum_v += pr->values[j];
        sum_absv += std::llabs((long long)pr->values[j]);
        max_w = std::max(max_w, pr->weights[j]);
        max_v = std::max(max_v, pr->values[j]);
        min_v = std::min(min_v, pr->values[j]);
    }
    const int64_t lim = (int64_t)1 << 62;
    if (sum_w >= lim / pa->penalty_lambda || sum_absv >= lim)
        return fail(QIEO_ERR_INVALID, "lambda * sum(w) or sum(|v|) reaches 2^62");

    qieo_instance *q = new (std::nothrow) qieo_instance();
    if (!q) return fail(QIEO_ERR_OOM, "host allocation failed");
    q->np = pa->np;
    q->ng = pr->ng;
    q->svec = (pr->ng + 7) / 8;
    q->xstride = (int32_t)align_up((size_t)q->svec, 16);
    q->D = pa->dtheta_den;
    q->K = pa->dtheta_den / 4;
    q->rule = pa->rotate_rule;
    q->host_de = pa->elite_on_host;
    q->flags = pa->flags;
    q->state8 = (pa->flags & QIEO_FLAG_STATE_I8) != 0;
    q->capacity = pr->capacity;
    q->lambda = pa->penalty_lambda;
    q->seed = pa->seed;
    q->inst_id = pa->instance_id;
    q->narrow_items = max_w <= 255 && max_v <= 255 && min_v >= 0;
    q->max_item = std::max(max_w, max_v);
    q->sum_w = sum_w;
    q->sum_v = sum_v;
    q->sum_absv = sum_absv;
    // elite key: fitness in [-lambda sum(w), sum(|v|)] must fit 40 bits, index 24 bits
    q->key_ok = sum_w < (((int64_t)1 << 39) / pa->penalty_lambda) &&
                sum_absv < ((int64_t)1 << 39) && q->np <= (1 << 24);

    auto bail = [&](qieo_status st) {
        qieo_destroy_instance(q);
        return st;
    };

    cudaError_t ce = cudaGetDevice(&q->device);
    if (ce != cudaSuccess) return bail(fail(QIEO_ERR_CUDA, "no CUDA device: %s", cudaGetErrorString(ce)));
    ce = cudaDeviceGetAttribute(&q->sm_count, cudaDevAttrMultiProcessorCount, q->device);
    if (ce != cudaSuccess) return bail(fail(QIEO_ERR_CUDA, "device query: %s", cudaGetErrorString(ce)));
    if (pa->stream) {
        q->stream = (cudaStream_t)pa->stream;
    } else {
        ce = cudaStreamCreateWithFlags(&q->stream, cudaStreamNonBlocking);
        if (ce != cudaSuccess) return bail(fail(QIEO_ERR_CUDA, "stream: %s", cudaGetErrorString(ce)));
        q->own_stream = true;
    }
    const size_t ngp = (size_t)q->svec * 8;
    size_t off[kParts];
    const size_t total = instance_layout(q->ng, q->np, q->D, ext ? ext->hist_cap : 0, off, q->state8);
    if (ext) {
        if (!ext->block || ext->bytes < total) return bail(fail(QIEO_ERR_INVALID, "placement too small"));
        q->block = ext->block;
        q->owns_block = false;
    } else {
        // stream-ordered allocation from the device's pool: no device-wide synchronisation
        // at allocation or release, and a freed block is reused by the next instance
        keep_pool_memory(q->device);
        ce = cudaMallocAsync(&q->block, total, q->stream);
        if (ce != cudaSuccess)
            return bail(fail(ce == cudaErrorMemoryAllocation ? QIEO_ERR_OOM : QIEO_ERR_CUDA,
                             "device allocation of %zu bytes: %s", total, cudaGetErrorString(ce)));
    }
    char *b = (char *)q->block;
    qieo::GenParams &g = q->gp;
    g.state = (uint4 *)(b + off[0]);
    g.state8 = q->state8 ? 1 : 0;
    g.xbits = (uint8_t *)(b + off[1]);
    q->items_narrow = (const uint4 *)(b + off[2]);
    g.w4 = (const int4 *)(b + off[3]);
    g.v4 = (const int4 *)(b + off[3] + ngp * 4);
    g.best_row = (uint8_t *)(b + off[4]);
    g.acc = (unsigned long long *)(b + off[5]);
    g.cnt = (unsigned int *)(b + off[6]);
    g.fitness = (int64_t *)(b + off[7]);
    g.best = (int64_t *)(b + off[8]);
    g.gen = (int32_t *)(b + off[9]);
    g.ticket = (unsigned int *)(b + off[10]);
    g.keys = (unsigned long long *)(b + off[11]);
    g.elite_idx = (int32_t *)(b + off[12]);
    g.thr = (const uint32_t *)(b + off[13]);
    g.bar_gen = (int32_t *)(b + off[14]);
    g.error = (int32_t *)(b + off[15]);
    g.conv = g.error + 1;
    g.qctr = reinterpret_cast<unsigned int *>(g.error + 5);
    g.converge = (q->flags & QIEO_FLAG_CONVERGE) ? 1 : 0;
    g.wait_ns = kDefaultBarrierWaitNs;
    g.np = q->np;
    g.svec = q->svec;
    g.xstride = q->xstride;
    g.xplane = (size_t)q->np * q->xstride;
    g.K = q->K;
    g.capacity = q->capacity;
    g.lambda = q->lambda;
    for (int r = 0; r < 10; ++r) {   // Philox key schedule: key + r * (Weyl increments)
        g.rk0[r] = q->seed + (uint32_t)r * qieo::kPhiloxW0;
        g.rk1[r] = q->inst_id + (uint32_t)r * qieo::kPhiloxW1;
    }

    // Items in both layouts, padded with zeros to whole vectors (padding adds nothing).
    // Narrow: (v << 16 | w) per gene, then per vector of 8 genes the byte vectors
    // (w0, w2, w1, w3), (w4, w6, w5, w7), (v0, v2, v1, v3), (v4, v6, v5, v7), in the byte
    // order the kernels build alleles in.
    std::vector<uint32_t> packed(ngp + ngp / 2, 0u), wide(2 * ngp, 0u);
    static const int kByteOf[8] = {0, 2, 1, 3, 0, 2, 1, 3};
    for (int32_t j = 0; j < q->ng; ++j) {
        if (q->narrow_items) {
            packed[(size_t)j] = ((uint32_t)pr->values[j] << 16) | (uint32_t)pr->weights[j];
            const size_t v = (size_t)j / 8;
            const int i = j % 8, hi = i / 4, sh = 8 * kByteOf[i];
            packed[ngp + 4 * v + hi] |= (uint32_t)pr->weights[j] << sh;
            packed[ngp + 4 * v + 2 + hi] |= (uint32_t)pr->values[j] << sh;
        }
        wide[(size_t)j] = (uint32_t)pr->weights[j];
        wide[ngp + (size_t)j] = (uint32_t)pr->values[j];
    }
    if (q->narrow_items) {   // per tile of 256 vectors (2,048 genes): the biases of sparse row changes
        const int32_t nt = (q->svec + qieo::kThreads - 1) / qieo::kThreads;
        q->tile_sums.assign((size_t)2 * nt, 0u);
        for (int32_t j = 0; j < q->ng; ++j) {
            q->tile_sums[(size_t)2 * (j / (8 * qieo::kThreads))] += (uint32_t)pr->weights[j];
            q->tile_sums[(size_t)2 * (j / (8 * qieo::kThreads)) + 1] += (uint32_t)pr->values[j];
        }
    }
    std::vector<uint64_t> T;
    build_thresholds(q->D, T);
    std::vector<uint32_t> T32(T.size());
    for (size_t i = 0; i < T.size(); ++i) T32[i] = (uint32_t)(T[i] & 0xffffffffull);

    // One copy for the items (both layouts) and the thresholds: the parts between them are
    // sent as zeros and set by the generation-0 initialisation that follows on the stream.
    {
        const size_t lo = off[2], hi = off[13] + T32.size() * 4;
        std::vector<char> stage(hi - lo, 0);
        std::memcpy(stage.data() + (off[2] - lo), packed.data(), packed.size() * 4);
        std::memcpy(stage.data() + (off[3] - lo), wide.data(), wide.size() * 4);
        std::memcpy(stage.data() + (off[13] - lo), T32.data(), T32.size() * 4);
        ce = cudaMemcpyAsync(b + lo, stage.data(), stage.size(), cudaMemcpyHostToDevice, q->stream);
        if (ce != cudaSuccess) return bail(fail(QIEO_ERR_CUDA, "upload: %s", cudaGetErrorString(ce)));
    }

    if (q->host_de) {
        ce = cudaMallocHost(&q->h_fit, (size_t)q->np * sizeof(int64_t));
        if (ce != cudaSuccess) return bail(fail(QIEO_ERR_OOM, "pinned host buffer: %s", cudaGetErrorString(ce)));
    }
    default_tile(q);
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tuned.find(TuneKey{q->ng, q->np, q->D, q->rule, q->narrow_items ? 1 : 0});
        if (it != g_tuned.end()) {
            q->lanes = it->second.first;
            q->warps = it->second.second;
        }
    }
    qieo_status st = configure(q);
    if (st != QIEO_OK) return bail(st);
    if (ext) {
        q->hist_e = (int32_t *)(b + off[16]);
        q->hist_f = (int64_t *)(b + off[17]);
        q->hist_cap = ext->hist_cap;
        q->fixed_history = true;
        q->gp.hist_e = q->hist_e;
        q->gp.hist_f = q->hist_f;
    } else {
        st = ensure_history(q, 1024);
        if (st != QIEO_OK) return bail(st);
    }
    st = qieo_reset(q);
    if (st != QIEO_OK) return bail(st);
    if (sync) {
        st = wait_stream(q->stream);
        if (st != QIEO_OK) return bail(st);
    }
    *out = q;
    return QIEO_OK;
}

}  // namespace

extern "C" {

qieo_status qieo_create_instance(const qieo_problem *pr, const qieo_params *pa,
                                 qieo_instance **out)
{
    return create_instance_impl(pr, pa, nullptr, true, out);
}

qieo_status qieo_destroy_instance(qieo_instance *q)
{
    if (!q) return QIEO_OK;
    cudaSetDevice(q->device);
    if (q->stream) cudaStreamSynchronize(q->stream);
    drop_graphs(q);
    if (q->block && q->owns_block) cudaFreeAsync(q->block, q->stream);
    if (q->hist_e && !q->fixed_history) cudaFreeAsync(q->hist_e, q->stream);
    if (q->hist_f && !q->fixed_history) cudaFreeAsync(q->hist_f, q->stream);
    if (q->segq) cudaFreeAsync(q->segq, q->stream);
    if (q->segq2) cudaFreeAsync(q->segq2, q->stream);
    if (q->ext_elite) cudaFreeAsync(q->ext_elite, q->stream);
    if (q->gen_ns) cudaFreeAsync(q->gen_ns, q->stream);
    if (q->fword_mem) cudaFreeAsync(q->fword_mem, q->stream);
    if (q->h_fit) cudaFreeHost(q->h_fit);
    if (q->ev0) cudaEventDestroy(q->ev0);
    if (q->ev1) cudaEventDestroy(q->ev1);
    for (cudaEvent_t e : q->phase_ev) cudaEventDestroy(e);
    for (cudaEvent_t e : q->gen_ev) cudaEventDestroy(e);
    if (q->own_stream && q->stream) {
        cudaStreamSynchronize(q->stream);   // the block's release is ordered on it
        cudaStreamDestroy(q->stream);
    }
    delete q;
    return QIEO_OK;
}

qieo_status qieo_reset(qieo_instance *q)
{
    qieo_status st = check_inst(q);
    if (st != QIEO_OK) return st;
    st = set_device(q);
    if (st != QIEO_OK) return st;
    const size_t words = (size_t)q->np * q->svec * (q->state8 ? 2 : 4);
    const size_t xbytes = 2 * (size_t)q->np * q->xstride;
    const int blocks = std::max(1, std::min(q->sm_count * 4, (int)((words + 255) / 256)));
    qieo::init_kernel<<<blocks, qieo::kThreads, 0, q->stream>>>(q->gp, words, xbytes,
                                                               (size_t)q->np * 2);
    CUDA_TRY(cudaGetLastError());
    if (q->hist_d)
        CUDA_TRY(cudaMemsetAsync(q->hist_d, 0, (size_t)q->hist_cap * sizeof(unsigned long long), q->stream));
    q->fword_dirty = false;   // init_kernel clears the words with the state
    q->t = 0;
    q->rows_t = -1;
    if (q->flags & QIEO_FLAG_SYNC_RUN) return wait_stream(q->stream);
    return QIEO_OK;
}

qieo_status qieo_run(qieo_instance *q, int32_t G)
{
    qieo_status st = check_inst(q);
    if (st != QIEO_OK) return st;
    if (G < 0) return fail(QIEO_ERR_INVALID, "generations must be >= 0 (got %d)", G);
    if (q->row_block)
        return fail(QIEO_ERR_INVALID, "a row block advances through qieo_rows_observe and qieo_rows_rotate");
    if (G == 0) return QIEO_OK;
    if ((int64_t)q->t + G > INT32_MAX / 2) return fail(QIEO_ERR_INVALID, "generation counter overflow");
    st = set_device(q);
    if (st != QIEO_OK) return st;
    st = ensure_history(q, q->t + G);
    if (st != QIEO_OK) return st;
    st = q->host_de ? run_host_de(q, G)
                    : (q->flags & QIEO_FLAG_UNFUSED) ? run_unfused(q, G) : run_device(q, G);
    if (st != QIEO_OK) return st;
    q->t += G;
    if (q->flags & QIEO_FLAG_SYNC_RUN) return wait_checked(q);
    return QIEO_OK;
}

qieo_status qieo_set_wait_timeout(qieo_instance *q, int64_t ns)
{
    qieo_status st = check_inst(q);
    if (st != QIEO_OK) return st;
    if (ns < 1) return fail(QIEO_ERR_INVALID, "wait timeout must be >= 1 ns");
    q->gp.wait_ns = (uint64_t)ns;
    drop_graphs(q);
    return QIEO_OK;
}

qieo_status qieo_synchronize(qieo_instance *q)
{
    qieo_status st = check_inst(q);
    if (st != QIEO_OK) return st;
    st = set_device(q);
    if (st != QIEO_OK) return st;
    return wait_checked(q);
}

namespace {

qieo_status fetch(qieo_instance *q, void *dst, const void *src, size_t bytes)
{
    qieo_status st = wait_checked(q);
    if (st != QIEO_OK) return st;
    CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, q->stream));
    return wait_stream(q->stream);
}

void unpack_row(const uint8_t *packed, int32_t ng, uint8_t *out)
{
    for (int32_t j = 0; j < ng; ++j) out[j] = (uint8_t)((packed[j >> 3] >> (j & 7)) & 1u);
}

}  // namespace

qieo_status qieo_get_best(qieo_instance *q, uint8_t *bits_out, int64_t *fitness,
                          int32_t *generation, int32_t *chromosome)
{
    qieo_status st = check_inst(q);
    if (st != QIEO_OK) return st;
    st = set_device(q);
    if (st != QIEO_OK) return st;
    // the error word, the record and the row in one round: copies into a pinned bounce
    // buffer queued behind the instance's work, one wait
    char *pin = nullptr;
    st = pinned_scratch(64 + (size_t)q->xstride, &pin);
    if (st != QIEO_OK) return st;
    int32_t *err_h = reinterpret_cast<int32_t *>(pin);
    int64_t *best_h = reinterpret_cast<int64_t *>(pin + 8);
    uint8_t *row_h = reinterpret_cast<uint8_t *>(pin + 64);
    CUDA_TRY(cudaMemcpyAsync(err_h, q->gp.error, sizeof(int32_t), cudaMemcpyDeviceToHost, q->stream));
    CUDA_TRY(cudaMemcpyAsync(best_h, q->gp.best, 3 * sizeof(int64_t), cudaMemcpyDeviceToHost, q->stream));
    if (bits_out)
        CUDA_TRY(cudaMemcpyAsync(row_h, q->gp.best_row, (size_t)q->xstride, cudaMemcpyDeviceToHost, q->stream));
    st = wait_stream(q->stream);
    if (st != QIEO_OK) return st;
    if (*err_h) return wait_checked(q);   // reports the recorded device error
    const int64_t best[3] = {best_h[0], best_h[1], best_h[2]};
    if (bits_out) unpack_row(row_h, q->ng, bits_out);
    if (fitness) *fitness = best[0];
    if (generation) *generation = (int32_t)best[1];
    if (chromosome) *chromosome = (int32_t)best[2];
    return QIEO_OK;
}

qieo_status qieo_get_state(qieo_instance *q, int16_t *k_out, int32_t *t_out)
{
    qieo_status st = check_inst(q);
    if (st != QIEO_OK) return st;
    st = set_device(q);
    if (st != QIEO_OK) return st;
    if (k_out && q->state8) {
        std::vector<uint8_t> s((size_t)q->np * q->svec * 8);
        st = fetch(q, s.data(), q->gp.state, s.size());
        if (st != QIEO_OK) return st;
        for (int32_t c = 0; c < q->np; ++c)
            for (int32_t j = 0; j < q->ng; ++j)
                k_out[(size_t)c * q->ng + j] =
                    (int16_t)((int32_t)(s[(size_t)c * q->svec * 8 + j] >> 2) - q->K);
    } else if (k_out) {
        std::vector<uint16_t> s((size_t)q->np * q->svec * 8);
        st = fetch(q, s.data(), q->gp.state, s.size() * 2);
        if (st != QIEO_OK) return st;
        for (int32_t c = 0; c < q->np; ++c)
            for (int32_t j = 0; j < q->ng; ++j)
                k_out[(size_t)c * q->ng + j] =
                    (int16_t)((int32_t)(s[(size_t)c * q->svec * 8 + j] >> 2) - q->K);
    }
    if (t_out) {
        int32_t t = 0;
        st = fetch(q, &t, q->gp.gen, sizeof t);
        if (st != QIEO_OK) return st;
        *t_out = t;
    }
    return QIEO_OK;
}

qieo_status qieo_get_fitness(qieo_instance *q, int64_t *f_out)
{
    qieo_status st = check_inst(q);
    if (st != QIEO_OK) return st;
    if (!f_out) return fail(QIEO_ERR_INVALID, "f_out is NULL");
    st = set_device(q);
    if (st != QIEO_OK) return st;
    return fetch(q, f_out, q->gp.fitness, (size_t)q->np * sizeof(int64_t));
}

qieo_status qieo_get_allele_row(qieo_instance *q, int32_t c, uint8_t *x_out)
{
    qieo_status st = check_inst(q);
    if (st != QIEO_OK) return st;
    if (!x_out) return fail(QIEO_ERR_INVALID, "x_out is NULL");
    if (c < 0 || c >= q->np) return fail(QIEO_ERR_INVALID, "chromosome %d outside [0, %d)", c, q->np);
    st = set_device(q);
    if (st != QIEO_OK) return st;
    std::vector<uint8_t> x((size_t)q->xstride);
    const uint8_t *row = q->gp.xbits + (size_t)((q->t + 1) & 1) * q->gp.xplane + (size_t)c * q->xstride;
    st = fetch(q, x.data(), row, x.size());
    if (st != QIEO_OK) return st;
    unpack_row(x.data(), q->ng, x_out);
    return QIEO_OK;
}

qieo_status qieo_get_alleles(qieo_instance *q, uint8_t *x_out)
{
    qieo_status st = check_inst(q);
    if (st != QIEO_OK) return st;
    if (!x_out) return fail(QIEO_ERR_INVALID, "x_out is NULL");
    st = set_device(q);
    if (st != QIEO_OK) return st;
    std::vector<uint8_t> x((size_t)q->np * q->xstride);
    const uint8_t *plane = q->gp.xbits + (size_t)((q->t + 1) & 1) * q->gp.xplane;
    st = fetch(q, x.data(), plane, x.size());
    if (st != QIEO_OK) return st;
    for (int32_t c = 0; c < q->np; ++c)
        unpack_row(x.data() + (size_t)c * q->xstride, q->ng, x_out + (size_t)c * q->ng);
    return QIEO_OK;
}

qieo_status qieo_get_elite_history(qieo_instance *q, int32_t first, int32_t n, int32_t *idx_out,
                                   int64_t *fit_out)
{
    qieo_status st = check_inst(q);
    if (st != QIEO_OK) return st;
    if (first < 0 || n < 0 || (int64_t)first + n > q->t)
        return fail(QIEO_ERR_INVALID, "history range [%d, %d) outside [0, %d)", first, first + n, q->t);
    if (n == 0) return QIEO_OK;
    st = set_device(q);
    if (st != QIEO_OK) return st;
    if (idx_out) {
        st = fetch(q, idx_out, q->hist_e + first, (size_t)n * sizeof(int32_t));
        if (st != QIEO_OK) return st;
    }
    if (fit_out) {
        st = fetch(q, fit_out, q->hist_f + first, (size_t)n * sizeof(int64_t));
        if (st != QIEO_OK) return st;
    }
    return QIEO_OK;
}

qieo_status qieo_get_drawn_vectors(qieo_instance *q, int32_t first, int32_t n, int64_t *out)
{
    qieo_status st = check_inst(q);
    if (st != QIEO_OK) return st;
    if (!out && n > 0) return fail(QIEO_ERR_INVALID, "out is NULL");
    if (!q->gp.fword || !q->hist_d)
        return fail(QIEO_ERR_INVALID, "the instance keeps no fixed-vector words (qieo_launch_shape.fixed_words)");
    if (first < 0 || n < 0 || (int64_t)first + n > q->t)
        return fail(QIEO_ERR_INVALID, "generation range [%d, %d) outside [0, %d)", first, first + n, q->t);
    if (n == 0) return QIEO_OK;
    st = set_device(q);
    if (st != QIEO_OK) return st;
    st = fetch(q, out, q->hist_d + first, (size_t)n * sizeof(int64_t));   // the vectors skipped
    if (st != QIEO_OK) return st;
    const int64_t all = (int64_t)q->np * q->svec;
    for (int32_t i = 0; i < n; ++i) out[i] = all - out[i];
    return QIEO_OK;
}

qieo_status qieo_get_threshold_table(qieo_instance *q, uint64_t *t_out)
{
    qieo_status st = check_inst(q);
    if (st != QIEO_OK) return st;
    if (!t_out) return fail(QIEO_ERR_INVALID, "t_out is NULL");
    st = set_device(q);
    if (st != QIEO_OK) return st;
    std::vector<uint32_t> T32((size_t)(2 * q->K + 1));
    st = fetch(q, T32.data(), q->gp.thr, T32.size() * 4);
    if (st != QIEO_OK) return st;
    for (size_t i = 0; i < T32.size(); ++i) t_out[i] = T32[i];
    t_out[2 * q->K] = 1ull << 32;   // stored as 0; the kernel treats n = 2K as "always 1"
    return QIEO_OK;
}

qieo_status qieo_get_launch_shape(qieo_instance *q, qieo_launch_shape *s)
{
    qieo_status st = check_inst(q);
    if (st != QIEO_OK) return st;
    if (!s) return fail(QIEO_ERR_INVALID, "shape is NULL");
    s->lanes_per_row = q->lanes;
    s->warps_per_row = q->warps;
    s->grid_ctas = q->grid;
    s->narrow = q->narrow;
    s->tiles = q->gp.ntile;
    s->rows_per_cta = q->gp.seg_rows_max;
    s->persistent = (use_resident(q) || use_cooperative(q)) ? 1 : 0;
    s->resident = use_resident(q) ? 1 : 0;
    s->fixed_words = q->gp.fword ? 1 : 0;
    return QIEO_OK;
}

qieo_status qieo_set_launch_shape(qieo_instance *q, const qieo_launch_shape *s)
{
    qieo_status st = check_inst(q);
    if (st != QIEO_OK) return st;
    if (!s) return fail(QIEO_ERR_INVALID, "shape is NULL");
    const int L = s->lanes_per_row, W = s->warps_per_row;
    if (L < 1 || L > 32 || (L & (L - 1)))
        return fail(QIEO_ERR_INVALID, "lanes_per_row must be a power of two in [1, 32]");
    if (W < 1 || W > 8 || (W & (W - 1)) || (W > 1 && L != 32))
        return fail(QIEO_ERR_INVALID, "warps_per_row must be 1, 2, 4 or 8 (>1 needs 32 lanes)");
    if (s->grid_ctas < 0 || s->grid_ctas > (1 << 20))
        return fail(QIEO_ERR_INVALID, "grid_ctas must be in [0, 2^20]");
    st = set_device(q);
    if (st != QIEO_OK) return st;
    q->lanes = L;
    q->warps = W;
    q->grid_override = s->grid_ctas;
    return configure(q);
}

qieo_status qieo_get_kernel_time(qieo_instance *q, double *ms, int64_t *launches)
{
    qieo_status st = check_inst(q);
    if (st != QIEO_OK) return st;
    if (ms) *ms = q->kernel_ms;
    if (launches) *launches = q->kernel_launches;
    return QIEO_OK;
}

qieo_status qieo_get_generation_times(qieo_instance *q, int32_t n, float *ms_out, int32_t *count)
{
    qieo_status st = check_inst(q);
    if (st != QIEO_OK) return st;
    if (!(q->flags & QIEO_FLAG_TIME_GENERATIONS))
        return fail(QIEO_ERR_INVALID, "the instance was not created with QIEO_FLAG_TIME_GENERATIONS");
    if (n < 0 || (n > 0 && !ms_out)) return fail(QIEO_ERR_INVALID, "n must be >= 0 with room in ms_out");
    st = set_device(q);
    if (st != QIEO_OK) return st;
    st = wait_stream(q->stream);
    if (st != QIEO_OK) return st;
    const int32_t m = std::min(n, q->gen_ev_n);
    if (q->gen_ns_last) {
        std::vector<unsigned long long> ns((size_t)m + 1);
        st = fetch(q, ns.data(), q->gen_ns, ns.size() * sizeof(unsigned long long));
        if (st != QIEO_OK) return st;
        for (int32_t i = 0; i < m; ++i) ms_out[i] = (float)((double)(ns[(size_t)i + 1] - ns[(size_t)i]) * 1e-6);
    } else {
        for (int32_t i = 0; i < m; ++i)
            CUDA_TRY(cudaEventElapsedTime(ms_out + i, q->gen_ev[(size_t)i], q->gen_ev[(size_t)i + 1]));
    }
    if (count) *count = m;
    return QIEO_OK;
}

// ---------------------------------------------------------------------------------------
// Row blocks of one population sharded by chromosome rows. A block observes and evaluates
// its rows with draws keyed by the global chromosome index and reports its lowest-index
// best row; the caller finds the population's elite across blocks (an all-reduce of the
// packed key and a broadcast of the elite's alleles) and passes the elite row back for the
// rotation. The generation kernel runs the observation (first-generation form: no CIP);
// the rotation is a separate launch toward the supplied row.
// ---------------------------------------------------------------------------------------
qieo_status qieo_create_row_block(const qieo_problem *problem, const qieo_params *params, int32_t row0,
                                  qieo_instance **out)
{
    if (out) *out = nullptr;
    if (!problem || !params || !out) return fail(QIEO_ERR_INVALID, "NULL argument");
    if (row0 < 0) return fail(QIEO_ERR_INVALID, "row0 must be >= 0 (got %d)", row0);
    if (params->np < 1 || (int64_t)row0 + params->np > (int64_t)INT32_MAX)
        return fail(QIEO_ERR_INVALID, "rows [row0, row0 + np) must lie in [0, 2^31 - 1)");
    if (params->elite_on_host ||
        (params->flags & (QIEO_FLAG_UNFUSED | QIEO_FLAG_COOPERATIVE | QIEO_FLAG_CONVERGE)))
        return fail(QIEO_ERR_INVALID, "a row block excludes elite_on_host, QIEO_FLAG_UNFUSED, "
                    "QIEO_FLAG_COOPERATIVE and QIEO_FLAG_CONVERGE");
    qieo_instance *q = nullptr;
    qieo_status st = qieo_create_instance(problem, params, &q);
    if (st != QIEO_OK) return st;
    if (!q->key_ok) {
        qieo_destroy_instance(q);
        return fail(QIEO_ERR_INVALID, "a row block needs fitness values that fit the packed elite key "
                    "(lambda * sum(w) and sum(|v|) below 2^39)");
    }
    q->row_block = true;
    q->gp.row0 = row0;
    st = configure(q);   // a row block keeps no fixed-vector words
    if (st != QIEO_OK) {
        qieo_destroy_instance(q);
        return st;
    }
    cudaError_t ce = cudaMallocAsync(&q->ext_elite, (size_t)q->xstride, q->stream);
    if (ce != cudaSuccess) {
        qieo_destroy_instance(q);
        return fail(QIEO_ERR_OOM, "elite row buffer: %s", cudaGetErrorString(ce));
    }
    drop_graphs(q);
    *out = q;
    return QIEO_OK;
}

qieo_status qieo_rows_observe(qieo_instance *q, int32_t t, int64_t *best_fitness, int32_t *best_row)
{
    qieo_status st = check_inst(q);
    if (st != QIEO_OK) return st;
    if (!q->row_block) return fail(QIEO_ERR_INVALID, "not a row block (qieo_create_row_block)");
    if (t < 0 || t > INT32_MAX / 2) return fail(QIEO_ERR_INVALID, "generation t out of range (got %d)", t);
    st = set_device(q);
    if (st != QIEO_OK) return st;
    // generation t keys its draws and selects its key slot; the slot and the segment-queue
    // counter of t start at zero
    char *h = nullptr;
    st = pinned_scratch(16, &h);
    if (st != QIEO_OK) return st;
    st = wait_stream(q->stream);   // the pinned buffer may still feed an earlier copy
    if (st != QIEO_OK) return st;
    const int32_t next = t + 1;
    std::memcpy(h, &t, sizeof t);
    std::memcpy(h + 4, &next, sizeof next);
    CUDA_TRY(cudaMemcpyAsync(q->gp.gen, h, sizeof t, cudaMemcpyHostToDevice, q->stream));
    CUDA_TRY(cudaMemsetAsync(q->gp.keys + (t % 3), 0, sizeof(unsigned long long), q->stream));
    CUDA_TRY(cudaMemsetAsync(q->gp.qctr + (t % 3), 0, sizeof(unsigned int), q->stream));
    CUDA_TRY(launch_gen(q, 0, 1, 0));
    // the generation counter then names the next generation, as after qieo_run
    CUDA_TRY(cudaMemcpyAsync(q->gp.gen, h + 4, sizeof next, cudaMemcpyHostToDevice, q->stream));
    CUDA_TRY(cudaMemcpyAsync(h + 8, q->gp.keys + (t % 3), sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                             q->stream));
    st = wait_checked(q);
    if (st != QIEO_OK) return st;
    unsigned long long key = 0;
    std::memcpy(&key, h + 8, sizeof key);
    const int32_t e = (int32_t)(0xffffffu - (uint32_t)(key & 0xffffffull));
    if (e < 0 || e >= q->np)
        return fail(QIEO_ERR_CUDA, "internal error: generation %d of the row block closed without a best row", t);
    q->t = t + 1;
    q->rows_t = t;
    if (best_fitness) *best_fitness = (int64_t)(key >> 24) - qieo::kKeyBias;
    if (best_row) *best_row = q->gp.row0 + e;
    return QIEO_OK;
}

qieo_status qieo_rows_rotate(qieo_instance *q, const uint8_t *elite_bits)
{
    qieo_status st = check_inst(q);
    if (st != QIEO_OK) return st;
    if (!q->row_block) return fail(QIEO_ERR_INVALID, "not a row block (qieo_create_row_block)");
    if (!elite_bits) return fail(QIEO_ERR_INVALID, "elite_bits is NULL");
    if (q->rows_t < 0) return fail(QIEO_ERR_INVALID, "no generation observed since creation or reset");
    st = set_device(q);
    if (st != QIEO_OK) return st;
    char *h = nullptr;
    st = pinned_scratch((size_t)q->xstride, &h);
    if (st != QIEO_OK) return st;
    st = wait_stream(q->stream);
    if (st != QIEO_OK) return st;
    std::memset(h, 0, (size_t)q->xstride);
    for (int32_t j = 0; j < q->ng; ++j) {
        if (elite_bits[j] > 1) return fail(QIEO_ERR_INVALID, "elite_bits[%d] = %d is not 0 or 1", j, elite_bits[j]);
        h[j >> 3] = (char)((unsigned char)h[j >> 3] | (unsigned char)(elite_bits[j] << (j & 7)));
    }
    CUDA_TRY(cudaMemcpyAsync(q->ext_elite, h, (size_t)q->xstride, cudaMemcpyHostToDevice, q->stream));
    const size_t total = (size_t)q->np * q->svec;
    const int blocks = (int)std::max<size_t>(
        1, std::min<size_t>((total + qieo::kThreads - 1) / qieo::kThreads, (size_t)std::max(q->sm_count, 1) * 8));
    if (q->rule) qieo::rows_cip_kernel<1><<<blocks, qieo::kThreads, 0, q->stream>>>(q->gp, q->rows_t, q->ext_elite);
    else qieo::rows_cip_kernel<0><<<blocks, qieo::kThreads, 0, q->stream>>>(q->gp, q->rows_t, q->ext_elite);
    CUDA_TRY(cudaGetLastError());
    return wait_checked(q);
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Checkpoint / resume: everything a later run reads, so that load + run(b) equals the
// uninterrupted run bit for bit (the draws are keyed by the absolute generation).
// ---------------------------------------------------------------------------------------
namespace {

struct CheckpointHeader {
    char magic[8];
    int32_t ng, np, D, rule;
    uint32_t seed, inst;
    int32_t state8, t;
    int64_t capacity, lambda;
    int32_t conv[4];
    int64_t best[3];
    int32_t elite_idx, xstride;
    uint64_t state_bytes;
};

const char kCheckpointMagic[8] = {'Q', 'I', 'E', 'O', 'C', 'K', 'P', '1'};

size_t state_bytes_of(const qieo_instance *q)
{
    return (size_t)q->np * q->svec * (q->state8 ? 8 : 16);
}

size_t checkpoint_bytes(const qieo_instance *q, int32_t t)
{
    return sizeof(CheckpointHeader) + (size_t)q->xstride + (size_t)t * (sizeof(int32_t) + sizeof(int64_t)) +
           state_bytes_of(q);
}

qieo_status upload(qieo_instance *q, void *dst, const void *src, size_t bytes)
{
    if (bytes == 0) return QIEO_OK;
    CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, q->stream));
    return wait_stream(q->stream);
}

}  // namespace

extern "C" {

qieo_status qieo_checkpoint_size(qieo_instance *q, size_t *bytes)
{
    qieo_status st = check_inst(q);
    if (st != QIEO_OK) return st;
    if (!bytes) return fail(QIEO_ERR_INVALID, "bytes is NULL");
    st = set_device(q);
    if (st != QIEO_OK) return st;
    int32_t t = 0;
    st = fetch(q, &t, q->gp.gen, sizeof t);
    if (st != QIEO_OK) return st;
    *bytes = checkpoint_bytes(q, t);
    return QIEO_OK;
}

qieo_status qieo_checkpoint_save(qieo_instance *q, void *buffer, size_t bytes)
{
    qieo_status st = check_inst(q);
    if (st != QIEO_OK) return st;
    if (!buffer) return fail(QIEO_ERR_INVALID, "buffer is NULL");
    st = set_device(q);
    if (st != QIEO_OK) return st;
    CheckpointHeader h;
    std::memset(&h, 0, sizeof h);
    std::memcpy(h.magic, kCheckpointMagic, sizeof h.magic);
    h.ng = q->ng;
    h.np = q->np;
    h.D = q->D;
    h.rule = q->rule;
    h.seed = q->seed;
    h.inst = q->inst_id;
    h.state8 = q->state8 ? 1 : 0;
    h.capacity = q->capacity;
    h.lambda = q->lambda;
    h.xstride = q->xstride;
    h.state_bytes = state_bytes_of(q);
    st = fetch(q, &h.t, q->gp.gen, sizeof h.t);
    if (st == QIEO_OK) st = fetch(q, h.conv, q->gp.conv, sizeof h.conv);
    if (st == QIEO_OK) st = fetch(q, h.best, q->gp.best, sizeof h.best);
    if (st == QIEO_OK) st = fetch(q, &h.elite_idx, q->gp.elite_idx, sizeof h.elite_idx);
    if (st != QIEO_OK) return st;
    if (bytes < checkpoint_bytes(q, h.t))
        return fail(QIEO_ERR_INVALID, "buffer of %zu bytes; the checkpoint needs %zu", bytes,
                    checkpoint_bytes(q, h.t));
    char *p = (char *)buffer;
    std::memcpy(p, &h, sizeof h);
    p += sizeof h;
    st = fetch(q, p, q->gp.best_row, (size_t)q->xstride);
    p += q->xstride;
    if (st == QIEO_OK && h.t > 0) st = fetch(q, p, q->hist_e, (size_t)h.t * sizeof(int32_t));
    p += (size_t)h.t * sizeof(int32_t);
    if (st == QIEO_OK && h.t > 0) st = fetch(q, p, q->hist_f, (size_t)h.t * sizeof(int64_t));
    p += (size_t)h.t * sizeof(int64_t);
    if (st == QIEO_OK) st = fetch(q, p, q->gp.state, h.state_bytes);
    return st;
}

qieo_status qieo_checkpoint_load(qieo_instance *q, const void *buffer, size_t bytes)
{
    qieo_status st = check_inst(q);
    if (st != QIEO_OK) return st;
    if (!buffer || bytes < sizeof(CheckpointHeader)) return fail(QIEO_ERR_INVALID, "buffer too small");
    CheckpointHeader h;
    std::memcpy(&h, buffer, sizeof h);
    if (std::memcmp(h.magic, kCheckpointMagic, sizeof h.magic) != 0)
        return fail(QIEO_ERR_INVALID, "not a QIEO checkpoint");
    if (h.ng != q->ng || h.np != q->np || h.D != q->D || h.rule != q->rule || h.seed != q->seed ||
        h.inst != q->inst_id || h.state8 != (q->state8 ? 1 : 0) || h.capacity != q->capacity ||
        h.lambda != q->lambda || h.xstride != q->xstride || h.state_bytes != state_bytes_of(q))
        return fail(QIEO_ERR_INVALID, "the checkpoint belongs to another problem or other params");
    if (h.t < 0 || bytes < checkpoint_bytes(q, h.t)) return fail(QIEO_ERR_INVALID, "truncated checkpoint");
    st = qieo_reset(q);
    if (st == QIEO_OK) st = wait_checked(q);
    if (st == QIEO_OK) st = ensure_history(q, std::max(h.t, 1));
    if (st != QIEO_OK) return st;
    const char *p = (const char *)buffer + sizeof h;
    st = upload(q, q->gp.best_row, p, (size_t)q->xstride);
    p += q->xstride;
    if (st == QIEO_OK) st = upload(q, q->hist_e, p, (size_t)h.t * sizeof(int32_t));
    p += (size_t)h.t * sizeof(int32_t);
    if (st == QIEO_OK) st = upload(q, q->hist_f, p, (size_t)h.t * sizeof(int64_t));
    p += (size_t)h.t * sizeof(int64_t);
    if (st == QIEO_OK) st = upload(q, q->gp.state, p, h.state_bytes);
    if (st == QIEO_OK) st = clear_fword(q, q->stream);   // the words of the reset state
    if (st == QIEO_OK) st = upload(q, q->gp.conv, h.conv, sizeof h.conv);
    if (st == QIEO_OK) st = upload(q, q->gp.best, h.best, sizeof h.best);
    if (st == QIEO_OK) st = upload(q, q->gp.elite_idx, &h.elite_idx, sizeof h.elite_idx);
    if (st == QIEO_OK) st = upload(q, q->gp.gen, &h.t, sizeof h.t);
    if (st == QIEO_OK) st = upload(q, q->gp.bar_gen, &h.t, sizeof h.t);
    if (st != QIEO_OK) return st;
    q->t = h.t;
    return QIEO_OK;
}

}  // extern "C"

extern "C" {

qieo_status qieo_get_convergence(qieo_instance *q, int32_t *stopped, int32_t *stable)
{
    qieo_status st = check_inst(q);
    if (st != QIEO_OK) return st;
    st = set_device(q);
    if (st != QIEO_OK) return st;
    int32_t w[4] = {0, 0, 0, 0}, t = 0;
    st = fetch(q, w, q->gp.conv, sizeof w);
    if (st == QIEO_OK) st = fetch(q, &t, q->gp.gen, sizeof t);
    if (st != QIEO_OK) return st;
    if (stopped) *stopped = w[2] != qieo::kRunning ? 1 : 0;
    if (stable) *stable = t > 0 ? w[(t - 1) & 1] : 0;
    return QIEO_OK;
}

qieo_status qieo_get_phase_times(qieo_instance *q, double ms[4], int64_t *generations)
{
    qieo_status st = check_inst(q);
    if (st != QIEO_OK) return st;
    if (ms)
        for (int i = 0; i < 4; ++i) ms[i] = q->phase_ms[i];
    if (generations) *generations = q->phase_gens;
    return QIEO_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Batches
// ---------------------------------------------------------------------------------------
struct qieo_batch {
    struct Group {
        bool narrow = false;
        int32_t rule = 0;
        std::vector<qieo_instance *> members;
        int32_t grid = 1;
        size_t smem = 0;
        int32_t seg_rows_max = 1;
        void *dev = nullptr;                        // params | segs | queue | inst_segs | done
        std::vector<qieo::GenParams> host_params;   // what is on the device
        qieo::BatchArgs args{};
        size_t done_bytes = 0;
    };
    bool persistent = false;   // runs are one cooperative launch per group (batch_run_kernel)
    std::vector<qieo_instance *> members;
    std::vector<Group> groups;
    int device = 0;
    cudaStream_t stream = nullptr;
    std::vector<cudaStream_t> other_streams;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::map<int32_t, cudaGraphExec_t> graphs;
    std::map<int32_t, int32_t> run_lengths_seen;
};

namespace {

void drop_batch_graphs(qieo_batch *b)
{
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
}

template <bool N, int R, bool C>
struct PickBatch {
    static void (*get())(qieo::BatchArgs) { return &qieo::batch_generation_kernel<N, R, C>; }
};

void (*batch_run_kernel_of(bool narrow, int rule))(qieo::BatchArgs, int32_t)
{
    if (narrow) return rule ? &qieo::batch_run_kernel<true, 1> : &qieo::batch_run_kernel<true, 0>;
    return rule ? &qieo::batch_run_kernel<false, 1> : &qieo::batch_run_kernel<false, 0>;
}

void (*batch_kernel_of(bool narrow, int rule, bool cip))(qieo::BatchArgs)
{
    if (narrow) {
        if (rule) return cip ? PickBatch<true, 1, true>::get() : PickBatch<true, 1, false>::get();
        return cip ? PickBatch<true, 0, true>::get() : PickBatch<true, 0, false>::get();
    }
    if (rule) return cip ? PickBatch<false, 1, true>::get() : PickBatch<false, 1, false>::get();
    return cip ? PickBatch<false, 0, true>::get() : PickBatch<false, 0, false>::get();
}

// Cuts the members' tile-rows into segments of about a quarter of a block's average share
// (by cost: active vectors per row plus a fixed per-row overhead) and orders them largest
// first for the kernel's segment queue.
void partition(const std::vector<qieo_instance *> &members, int grid,
               std::vector<qieo::BatchSeg> &segs, std::vector<int32_t> &inst_segs,
               int32_t &seg_rows_max)
{
    struct Cut {
        qieo::BatchSeg seg;
        double cost;
    };
    // one pass covers rpp rows of a tile; its cost is the block's 256 thread-slots, of
    // which the ragged last tile of a row leaves some idle
    auto row_cost = [](const qieo_instance *q, int tile) {
        const int tv = q->lanes * q->warps;
        const int active = std::min(tv, q->svec - tile * tv);
        return (double)qieo::kThreads * (0.25 + 0.75 * (double)active / tv) / (qieo::kThreads / tv);
    };
    double total = 0.0;
    for (const qieo_instance *q : members) {
        const int tv = q->lanes * q->warps;
        const int ntile = (q->svec + tv - 1) / tv;
        for (int tile = 0; tile < ntile; ++tile) total += row_cost(q, tile) * q->np;
    }
    // About four segments per block on average: enough for the queue to even out the
    // blocks' loads, few enough that the per-segment flush stays small.
    const double target = std::max(1.0, total / (4.0 * grid));
    std::vector<Cut> cuts;
    inst_segs.assign(members.size(), 0);
    seg_rows_max = 1;
    for (size_t i = 0; i < members.size(); ++i) {
        const qieo_instance *q = members[i];
        const int tv = q->lanes * q->warps;
        const int rpp = qieo::kThreads / tv;
        const int ntile = (q->svec + tv - 1) / tv;
        const int max_rows = std::max(rpp, qieo::kMaxSegRows / rpp * rpp);
        for (int tile = 0; tile < ntile; ++tile) {
            const double rc = row_cost(q, tile);
            int want = (int)std::min<double>(max_rows, std::max<double>(rpp, target / rc));
            want = std::max(rpp, want / rpp * rpp);
            const int nseg = (q->np + want - 1) / want;
            int rows = (q->np + nseg - 1) / nseg;
            rows = std::min(max_rows, (rows + rpp - 1) / rpp * rpp);
            for (int ra = 0; ra < q->np; ra += rows) {
                const int r = std::min(rows, q->np - ra);
                cuts.push_back({{(int32_t)i, tile, ra, r}, rc * r});
                inst_segs[i] += 1;
                seg_rows_max = std::max(seg_rows_max, r);
            }
        }
    }
    std::stable_sort(cuts.begin(), cuts.end(), [](const Cut &x, const Cut &y) { return x.cost > y.cost; });
    segs.clear();
    segs.reserve(cuts.size());
    for (const Cut &c : cuts) segs.push_back(c.seg);
}

qieo_status upload_group(qieo_batch *bt, qieo_batch::Group &g)
{
    std::vector<qieo::GenParams> params;
    for (qieo_instance *q : g.members) params.push_back(q->gp);
    if (g.dev && params.size() == g.host_params.size() &&
        std::memcmp(params.data(), g.host_params.data(), params.size() * sizeof(qieo::GenParams)) == 0)
        return QIEO_OK;
    CUDA_TRY(cudaMemcpyAsync(const_cast<qieo::GenParams *>(g.args.params), params.data(),
                             params.size() * sizeof(qieo::GenParams), cudaMemcpyHostToDevice,
                             bt->stream));
    g.host_params = params;
    drop_batch_graphs(bt);
    return QIEO_OK;
}

qieo_status build_group(qieo_batch *bt, qieo_batch::Group &g)
{
    const qieo_instance *q0 = g.members[0];
    const size_t row_bytes = g.narrow ? 8 : 16;
    auto fn = batch_kernel_of(g.narrow, g.rule, true);
    auto fn0 = batch_kernel_of(g.narrow, g.rule, false);
    auto fr = batch_run_kernel_of(g.narrow, g.rule);
    const size_t smem_max = qieo::kRingBytes + (size_t)qieo::kMaxSegRows * row_bytes;
    for (auto f : {fn, fn0})
        CUDA_TRY(cudaFuncSetAttribute(reinterpret_cast<const void *>(f),
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max));
    CUDA_TRY(cudaFuncSetAttribute(reinterpret_cast<const void *>(fr),
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max));
    int bps = 0, bps_run = 0;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, reinterpret_cast<const void *>(fn),
                                                           qieo::kThreads, smem_max));
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps_run, reinterpret_cast<const void *>(fr),
                                                           qieo::kThreads, smem_max));
    // the persistent form needs every block resident at once
    if (bt->persistent) bps = std::min(bps, bps_run);
    if (bt->persistent && bps < 1) bt->persistent = false;
    g.grid = std::max(1, bps) * std::max(1, q0->sm_count);
    std::vector<qieo::BatchSeg> segs;
    std::vector<int32_t> inst_segs;
    partition(g.members, g.grid, segs, inst_segs, g.seg_rows_max);
    g.smem = qieo::kRingBytes + (size_t)g.seg_rows_max * row_bytes;
    const size_t n = g.members.size();
    size_t off[5], total = 0;
    const size_t sizes[5] = {n * sizeof(qieo::GenParams), segs.size() * sizeof(qieo::BatchSeg),
                             2 * sizeof(unsigned int), n * sizeof(int32_t), n * sizeof(unsigned int)};
    for (int i = 0; i < 5; ++i) {
        off[i] = total;
        total = align_up(total + sizes[i], 256);
    }
    CUDA_TRY(cudaMalloc(&g.dev, total));
    char *d = (char *)g.dev;
    g.args.params = (const qieo::GenParams *)(d + off[0]);
    g.args.segs = (const qieo::BatchSeg *)(d + off[1]);
    g.args.queue = (unsigned int *)(d + off[2]);
    g.args.inst_segs = (const int32_t *)(d + off[3]);
    g.args.done = (unsigned int *)(d + off[4]);
    g.done_bytes = sizes[4];
    g.args.nsegs = (int32_t)segs.size();
    g.args.seg_rows_max = g.seg_rows_max;
    CUDA_TRY(cudaMemcpyAsync(d + off[1], segs.data(), sizes[1], cudaMemcpyHostToDevice, bt->stream));
    CUDA_TRY(cudaMemsetAsync(d + off[2], 0, sizes[2], bt->stream));
    CUDA_TRY(cudaMemcpyAsync(d + off[3], inst_segs.data(), sizes[3], cudaMemcpyHostToDevice, bt->stream));
    qieo_status st = upload_group(bt, g);
    if (st != QIEO_OK) return st;
    return wait_stream(bt->stream);
}

// A persistent-form run: per group, the run's first generation (no CIP) as one batched
// launch, then the run-local close counters cleared and one cooperative launch for the
// other G - 1 generations (split so that generations x segments stays within 32 bits), and
// the final rotation.
qieo_status enqueue_batch_persistent(qieo_batch *bt, int32_t G)
{
    for (auto &g : bt->groups) {
        {
            cudaLaunchConfig_t cfg0 = {};
            cfg0.gridDim = dim3(g.grid);
            cfg0.blockDim = dim3(qieo::kThreads);
            cfg0.dynamicSmemBytes = g.smem;
            cfg0.stream = bt->stream;
            CUDA_TRY(cudaLaunchKernelEx(&cfg0, batch_kernel_of(g.narrow, g.rule, false), g.args));
        }
        const int32_t rest = G - 1;
        const int32_t chunk = (int32_t)std::max<int64_t>(1, std::min<int64_t>(std::max(rest, 1),
                                                                               ((int64_t)1 << 30) / std::max(1, g.args.nsegs)));
        for (int32_t done = 0; done < rest; done += chunk) {
            const int32_t n = std::min(chunk, rest - done);
            CUDA_TRY(cudaMemsetAsync(g.args.done, 0, g.done_bytes, bt->stream));
            cudaLaunchAttribute attr[1];
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(g.grid);
            cfg.blockDim = dim3(qieo::kThreads);
            cfg.dynamicSmemBytes = g.smem;
            cfg.stream = bt->stream;
            attr[0].id = cudaLaunchAttributeCooperative;
            attr[0].val.cooperative = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            CUDA_TRY(cudaLaunchKernelEx(&cfg, batch_run_kernel_of(g.narrow, g.rule), g.args, n));
        }
        if (g.rule) qieo::batch_cip_kernel<1><<<g.grid, qieo::kThreads, 0, bt->stream>>>(g.args);
        else qieo::batch_cip_kernel<0><<<g.grid, qieo::kThreads, 0, bt->stream>>>(g.args);
        CUDA_TRY(cudaGetLastError());
    }
    return QIEO_OK;
}

qieo_status enqueue_batch_run(qieo_batch *bt, int32_t G)
{
    for (int32_t gen = 0; gen < G; ++gen) {
        for (auto &g : bt->groups) {
            cudaLaunchAttribute attr[1];
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(g.grid);
            cfg.blockDim = dim3(qieo::kThreads);
            cfg.dynamicSmemBytes = g.smem;
            cfg.stream = bt->stream;
            attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            attr[0].val.programmaticStreamSerializationAllowed = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            CUDA_TRY(cudaLaunchKernelEx(&cfg, batch_kernel_of(g.narrow, g.rule, gen > 0), g.args));
        }
    }
    for (auto &g : bt->groups) {
        if (g.rule) qieo::batch_cip_kernel<1><<<g.grid, qieo::kThreads, 0, bt->stream>>>(g.args);
        else qieo::batch_cip_kernel<0><<<g.grid, qieo::kThreads, 0, bt->stream>>>(g.args);
        CUDA_TRY(cudaGetLastError());
    }
    return QIEO_OK;
}

}  // namespace

extern "C" {

qieo_status qieo_create_batch(qieo_instance *const *instances, int32_t n, qieo_batch **out)
{
    if (out) *out = nullptr;
    if (!instances || n < 1 || !out) return fail(QIEO_ERR_INVALID, "bad arguments");
    std::vector<qieo_instance *> members(instances, instances + n);
    for (int32_t i = 0; i < n; ++i) {
        if (!members[(size_t)i]) return fail(QIEO_ERR_INVALID, "instance %d is NULL", i);
        if (members[(size_t)i]->host_de)
            return fail(QIEO_ERR_INVALID, "instance %d uses elite_on_host; batches pick the elite on the device", i);
        if (members[(size_t)i]->state8)
            return fail(QIEO_ERR_INVALID, "instance %d stores its state as bytes; batches use 16-bit state", i);
        if (members[(size_t)i]->row_block)
            return fail(QIEO_ERR_INVALID, "instance %d is a row block of a sharded population", i);
        if (members[(size_t)i]->device != members[0]->device)
            return fail(QIEO_ERR_INVALID, "instance %d is on another device", i);
        for (int32_t j = 0; j < i; ++j)
            if (members[(size_t)j] == members[(size_t)i]) return fail(QIEO_ERR_INVALID, "instance %d repeats", i);
    }
    qieo_batch *bt = new (std::nothrow) qieo_batch();
    if (!bt) return fail(QIEO_ERR_OOM, "host allocation failed");
    bt->members = members;
    bt->device = members[0]->device;
    bt->stream = members[0]->stream;
    for (qieo_instance *q : members)
        if (q->stream != bt->stream &&
            std::find(bt->other_streams.begin(), bt->other_streams.end(), q->stream) == bt->other_streams.end())
            bt->other_streams.push_back(q->stream);
    auto bail = [&](qieo_status st) {
        qieo_destroy_batch(bt);
        return st;
    };
    cudaError_t ce = cudaSetDevice(bt->device);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&bt->ev_in, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&bt->ev_out, cudaEventDisableTiming);
    if (ce != cudaSuccess) return bail(fail(QIEO_ERR_CUDA, "batch setup: %s", cudaGetErrorString(ce)));
    // One persistent launch per run unless a member asks for one launch per generation or
    // uses the convergence test.
    bt->persistent = true;
    for (qieo_instance *q : members)
        if (q->flags & (QIEO_FLAG_CONVERGE | QIEO_FLAG_PER_GENERATION)) bt->persistent = false;
    for (qieo_instance *q : members) {
        auto it = std::find_if(bt->groups.begin(), bt->groups.end(), [&](const qieo_batch::Group &g) {
            return g.narrow == (q->narrow != 0) && g.rule == q->rule;
        });
        if (it == bt->groups.end()) {
            bt->groups.emplace_back();
            bt->groups.back().narrow = q->narrow != 0;
            bt->groups.back().rule = q->rule;
            it = bt->groups.end() - 1;
        }
        it->members.push_back(q);
    }
    for (auto &g : bt->groups) {
        qieo_status st = build_group(bt, g);
        if (st != QIEO_OK) return bail(st);
    }
    *out = bt;
    return QIEO_OK;
}

qieo_status qieo_destroy_batch(qieo_batch *bt)
{
    if (!bt) return QIEO_OK;
    cudaSetDevice(bt->device);
    if (bt->stream) cudaStreamSynchronize(bt->stream);
    drop_batch_graphs(bt);
    for (auto &g : bt->groups)
        if (g.dev) cudaFree(g.dev);
    if (bt->ev_in) cudaEventDestroy(bt->ev_in);
    if (bt->ev_out) cudaEventDestroy(bt->ev_out);
    delete bt;
    return QIEO_OK;
}

qieo_status qieo_batch_run(qieo_batch *bt, int32_t G)
{
    if (!bt) return fail(QIEO_ERR_INVALID, "batch is NULL");
    if (G < 0) return fail(QIEO_ERR_INVALID, "generations must be >= 0 (got %d)", G);
    if (G == 0) return QIEO_OK;
    CUDA_TRY(cudaSetDevice(bt->device));
    for (qieo_instance *q : bt->members) {
        if ((int64_t)q->t + G > INT32_MAX / 2) return fail(QIEO_ERR_INVALID, "generation counter overflow");
        qieo_status st = ensure_history(q, q->t + G);
        if (st != QIEO_OK) return st;
    }
    for (auto &g : bt->groups) {
        qieo_status st = upload_group(bt, g);
        if (st != QIEO_OK) return st;
    }
    for (cudaStream_t s : bt->other_streams) {   // pending work of the members' own streams
        CUDA_TRY(cudaEventRecord(bt->ev_in, s));
        CUDA_TRY(cudaStreamWaitEvent(bt->stream, bt->ev_in, 0));
    }
    const bool first_time = bt->run_lengths_seen[G]++ == 0;
    if (bt->persistent) {
        qieo_status st = enqueue_batch_persistent(bt, G);
        if (st != QIEO_OK) return st;
    } else if (first_time && !bt->graphs.count(G)) {
        qieo_status st = enqueue_batch_run(bt, G);
        if (st != QIEO_OK) return st;
    } else {
        auto it = bt->graphs.find(G);
        cudaGraphExec_t exec = nullptr;
        if (it == bt->graphs.end()) {
            if (bt->graphs.size() >= 8) drop_batch_graphs(bt);
            cudaGraph_t graph = nullptr;
            CUDA_TRY(cudaStreamBeginCapture(bt->stream, cudaStreamCaptureModeThreadLocal));
            qieo_status st = enqueue_batch_run(bt, G);
            cudaError_t ce = cudaStreamEndCapture(bt->stream, &graph);
            if (st != QIEO_OK) {
                if (graph) cudaGraphDestroy(graph);
                return st;
            }
            if (ce != cudaSuccess) return fail(QIEO_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ce));
            ce = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ce != cudaSuccess) return fail(QIEO_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ce));
            bt->graphs[G] = exec;
        } else {
            exec = it->second;
        }
        CUDA_TRY(cudaGraphLaunch(exec, bt->stream));
    }
    for (qieo_instance *q : bt->members) {   // the batched kernels do not keep F
        qieo_status st = clear_fword(q, bt->stream);
        if (st != QIEO_OK) return st;
    }
    if (!bt->other_streams.empty()) {
        CUDA_TRY(cudaEventRecord(bt->ev_out, bt->stream));
        for (cudaStream_t s : bt->other_streams) CUDA_TRY(cudaStreamWaitEvent(s, bt->ev_out, 0));
    }
    for (qieo_instance *q : bt->members) q->t += G;
    return QIEO_OK;
}

qieo_status qieo_autotune(qieo_instance *q, int32_t trials, qieo_launch_shape *shape_out)
{
    qieo_status st = check_inst(q);
    if (st != QIEO_OK) return st;
    if (trials < 1 || trials > 1000) return fail(QIEO_ERR_INVALID, "trial_generations must be in [1, 1000]");
    if (q->host_de) return fail(QIEO_ERR_INVALID, "autotune times the device path; elite_on_host is set");
    st = set_device(q);
    if (st != QIEO_OK) return st;
    st = ensure_events(q);
    if (st != QIEO_OK) return st;
    std::vector<std::pair<int, int>> cands;
    const int span = pow2_ceil(q->svec);
    for (int L = 1; L <= 16; L *= 2)
        if (L <= 2 * span) cands.push_back({L, 1});
    for (int W = 1; W <= 8; W *= 2)
        if (32 * W <= 2 * span || W == 1) cands.push_back({32, W});
    const int old_lanes = q->lanes, old_warps = q->warps, old_grid = q->grid_override;
    const int old_flags = q->flags;
    q->flags &= ~(QIEO_FLAG_TIME_KERNELS | QIEO_FLAG_SYNC_RUN);
    float best_ms = 1e30f;
    std::pair<int, int> best = {old_lanes, old_warps};
    for (const auto &c : cands) {
        q->lanes = c.first;
        q->warps = c.second;
        q->grid_override = 0;
        st = configure(q);
        if (st != QIEO_OK) break;
        float ms_min = 1e30f;
        for (int rep = 0; rep < 2 && st == QIEO_OK; ++rep) {
            st = qieo_reset(q);
            if (st != QIEO_OK) break;
            CUDA_TRY(cudaEventRecord(q->ev0, q->stream));
            st = run_device(q, trials);
            if (st != QIEO_OK) break;
            CUDA_TRY(cudaEventRecord(q->ev1, q->stream));
            st = wait_checked(q);
            if (st != QIEO_OK) break;
            float ms = 0.f;
            CUDA_TRY(cudaEventElapsedTime(&ms, q->ev0, q->ev1));
            ms_min = std::min(ms_min, ms);
        }
        if (st != QIEO_OK) break;
        if (ms_min < best_ms) {
            best_ms = ms_min;
            best = c;
        }
    }
    q->flags = old_flags;
    q->lanes = best.first;
    q->warps = best.second;
    q->grid_override = old_grid;
    qieo_status st2 = configure(q);
    if (st == QIEO_OK) st = st2;
    qieo_status st3 = qieo_reset(q);
    if (st == QIEO_OK) st = st3;
    q->run_lengths_seen.clear();
    if (st != QIEO_OK) return st;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tuned[TuneKey{q->ng, q->np, q->D, q->rule, q->narrow_items ? 1 : 0}] = best;
    }
    if (shape_out) return qieo_get_launch_shape(q, shape_out);
    return QIEO_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Serving
// ---------------------------------------------------------------------------------------
namespace {

// First-fit allocator over the arena (byte offsets) with a coalescing free list.
class ArenaAlloc {
  public:
    void init(size_t bytes)
    {
        free_.clear();
        free_[0] = bytes;
        total_ = bytes;
    }
    bool alloc(size_t bytes, size_t *off)
    {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            const size_t rest = it->second - bytes, noff = it->first + bytes;
            free_.erase(it);
            if (rest) free_[noff] = rest;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t total() const { return total_; }

  private:
    std::map<size_t, size_t> free_;
    size_t total_ = 0;
};

struct SolveRequest {
    int64_t id = 0;
    std::vector<int32_t> w, v;
    qieo_problem prob{};
    qieo_params params{};
    int32_t gens = 0;
    int32_t state = QIEO_SOLVE_QUEUED;
    int32_t status = QIEO_OK;
    double t_submit = 0, t_admit = 0, t_done = 0;
    qieo_instance *inst = nullptr;
    size_t off = 0, bytes = 0;
    int32_t remaining = 0;
    int64_t best[3] = {0, -1, -1};
    std::vector<uint8_t> best_row;
    int32_t gens_run = 0, converged = 0;
};

struct StepRecord {
    cudaEvent_t done = nullptr;
    std::vector<SolveRequest *> finishing;
    std::vector<SolveRequest *> watched;       // solves with the convergence test ...
    const int32_t *stop_host = nullptr;        // ... and their stop states after the step
};

constexpr size_t kWorkListBytes = 16u << 20;   // per region: params, segments, block starts

}  // namespace

struct qieo_server {
    qieo_server_config cfg{};
    int device = 0, sm_count = 0;
    cudaStream_t stream = nullptr, copy_stream = nullptr;
    char *arena = nullptr;
    ArenaAlloc alloc;
    char *wl_dev[2] = {nullptr, nullptr};
    char *wl_host[2] = {nullptr, nullptr};
    int wl_next = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::deque<SolveRequest *> queue;
    std::vector<SolveRequest *> active;
    std::unordered_map<int64_t, std::unique_ptr<SolveRequest>> all;
    std::deque<StepRecord> inflight;
    std::vector<cudaEvent_t> spare_events;
    int64_t next_id = 1;
    std::chrono::steady_clock::time_point t0;
    std::thread worker;
    int bps[2] = {1, 1};                 // batch kernel blocks per SM: [wide, narrow]
    int64_t n_submitted = 0, n_admitted = 0, n_completed = 0, n_steps = 0, n_launches = 0;
    int32_t max_active_seen = 0;
};

namespace {

double server_now(const qieo_server *S)
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - S->t0).count();
}

void destroy_instance_nosync(qieo_instance *q)
{
    drop_graphs(q);
    if (q->ev0) cudaEventDestroy(q->ev0);
    if (q->ev1) cudaEventDestroy(q->ev1);
    for (cudaEvent_t e : q->phase_ev) cudaEventDestroy(e);
    delete q;
}

// Enqueues `G` generations (+ the final rotation) of every member on the server stream
// with the batched kernel; the work list goes through the next double-buffered region.
qieo_status enqueue_server_step(qieo_server *S, const std::vector<qieo_instance *> &members, int32_t G,
                                int64_t *launched, const std::vector<qieo_instance *> &watch,
                                const int32_t **stop_host)
{
    *launched = 0;
    *stop_host = nullptr;
    const int r = S->wl_next;
    S->wl_next ^= 1;
    char *host = S->wl_host[r];
    char *dev = S->wl_dev[r];
    size_t used = 0;
    struct Launch {
        bool narrow;
        int rule;
        int grid;
        size_t smem;
        qieo::BatchArgs args;
    };
    std::vector<Launch> launches;
    for (int narrow = 0; narrow < 2; ++narrow) {
        for (int rule = 0; rule < 2; ++rule) {
            std::vector<qieo_instance *> grp;
            for (qieo_instance *q : members)
                if (q->narrow == narrow && q->rule == rule) grp.push_back(q);
            if (grp.empty()) continue;
            const int grid = S->bps[narrow] * S->sm_count;
            std::vector<qieo::BatchSeg> segs;
            std::vector<int32_t> inst_segs;
            int32_t seg_rows_max = 1;
            partition(grp, grid, segs, inst_segs, seg_rows_max);
            const size_t sizes[4] = {grp.size() * sizeof(qieo::GenParams), segs.size() * sizeof(qieo::BatchSeg),
                                     2 * sizeof(unsigned int), inst_segs.size() * sizeof(int32_t)};
            size_t off[4];
            for (int i = 0; i < 4; ++i) {
                off[i] = used;
                used = align_up(used + sizes[i], 256);
            }
            if (used > kWorkListBytes)
                return fail(QIEO_ERR_INVALID, "too many resident solves for one work list");
            for (size_t i = 0; i < grp.size(); ++i)
                std::memcpy(host + off[0] + i * sizeof(qieo::GenParams), &grp[i]->gp, sizeof(qieo::GenParams));
            std::memcpy(host + off[1], segs.data(), sizes[1]);
            std::memset(host + off[2], 0, sizes[2]);   // the segment queue starts empty
            std::memcpy(host + off[3], inst_segs.data(), sizes[3]);
            Launch L;
            L.narrow = narrow != 0;
            L.rule = rule;
            L.grid = grid;
            L.smem = qieo::kRingBytes + (size_t)seg_rows_max * (narrow ? 8 : 16);
            L.args.params = (const qieo::GenParams *)(dev + off[0]);
            L.args.segs = (const qieo::BatchSeg *)(dev + off[1]);
            L.args.queue = (unsigned int *)(dev + off[2]);
            L.args.inst_segs = (const int32_t *)(dev + off[3]);
            L.args.nsegs = (int32_t)segs.size();
            L.args.seg_rows_max = seg_rows_max;
            launches.push_back(L);
        }
    }
    CUDA_TRY(cudaMemcpyAsync(dev, host, used, cudaMemcpyHostToDevice, S->stream));
    for (int32_t gen = 0; gen < G; ++gen) {
        for (const Launch &L : launches) {
            cudaLaunchAttribute attr[1];
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(L.grid);
            cfg.blockDim = dim3(qieo::kThreads);
            cfg.dynamicSmemBytes = L.smem;
            cfg.stream = S->stream;
            attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            attr[0].val.programmaticStreamSerializationAllowed = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            CUDA_TRY(cudaLaunchKernelEx(&cfg, batch_kernel_of(L.narrow, L.rule, gen > 0), L.args));
        }
    }
    for (const Launch &L : launches) {
        if (L.rule) qieo::batch_cip_kernel<1><<<L.grid, qieo::kThreads, 0, S->stream>>>(L.args);
        else qieo::batch_cip_kernel<0><<<L.grid, qieo::kThreads, 0, S->stream>>>(L.args);
        CUDA_TRY(cudaGetLastError());
    }
    *launched = (int64_t)launches.size() * (G + 1);
    if (!watch.empty()) {   // stop states of the solves with the convergence test, to the host
        const size_t nw = watch.size();
        const size_t p_off = used, o_off = align_up(p_off + nw * sizeof(int32_t *), 256);
        const size_t end = align_up(o_off + nw * sizeof(int32_t), 256);
        if (end > kWorkListBytes) return fail(QIEO_ERR_INVALID, "too many resident solves for one work list");
        for (size_t i = 0; i < nw; ++i) std::memcpy(host + p_off + i * sizeof(int32_t *), &watch[i]->gp.conv, sizeof(int32_t *));
        CUDA_TRY(cudaMemcpyAsync(dev + p_off, host + p_off, nw * sizeof(int32_t *), cudaMemcpyHostToDevice, S->stream));
        const int blocks = (int)std::min<size_t>(64, (nw + qieo::kThreads - 1) / qieo::kThreads);
        qieo::gather_stop_kernel<<<blocks, qieo::kThreads, 0, S->stream>>>(
            (int32_t *const *)(dev + p_off), (int32_t)nw, (int32_t *)(dev + o_off));
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaMemcpyAsync(host + o_off, dev + o_off, nw * sizeof(int32_t), cudaMemcpyDeviceToHost, S->stream));
        *stop_host = (const int32_t *)(host + o_off);
        *launched += 1;
    }
    return QIEO_OK;
}

// Results of the solves that finished with the oldest step in flight.
void retire_oldest_step(qieo_server *S)
{
    StepRecord rec = S->inflight.front();
    S->inflight.pop_front();
    const auto t_wait = std::chrono::steady_clock::now();
    cudaError_t ce;
    while ((ce = cudaEventQuery(rec.done)) == cudaErrorNotReady) {
        if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t_wait).count() > kWaitSeconds)
            break;
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    const qieo_status step_st = ce == cudaSuccess ? QIEO_OK : (ce == cudaErrorNotReady ? QIEO_ERR_TIMEOUT : QIEO_ERR_CUDA);
    // Solves that converged in this step leave the resident set now; their memory is
    // released once the step already queued after this one (which includes them but does
    // nothing for a stopped solve) has finished too.
    if (step_st == QIEO_OK && rec.stop_host) {
        std::lock_guard<std::mutex> lock(S->mu);
        for (size_t i = 0; i < rec.watched.size(); ++i) {
            SolveRequest *R = rec.watched[i];
            if (rec.stop_host[i] != qieo::kStopped) continue;
            auto it = std::find(S->active.begin(), S->active.end(), R);
            if (it == S->active.end()) continue;   // already finishing by its generation count
            S->active.erase(it);
            R->converged = 1;
            R->remaining = 0;
            if (!S->inflight.empty()) S->inflight.back().finishing.push_back(R);
            else rec.finishing.push_back(R);
        }
    }
    for (SolveRequest *R : rec.finishing) {
        qieo_instance *q = R->inst;
        int32_t st = step_st;
        if (st == QIEO_OK) {
            R->best_row.resize((size_t)q->xstride);
            if (cudaMemcpyAsync(R->best, q->gp.best, sizeof R->best, cudaMemcpyDeviceToHost, S->copy_stream) != cudaSuccess ||
                cudaMemcpyAsync(&R->gens_run, q->gp.gen, sizeof R->gens_run, cudaMemcpyDeviceToHost,
                                S->copy_stream) != cudaSuccess ||
                cudaMemcpyAsync(R->best_row.data(), q->gp.best_row, R->best_row.size(), cudaMemcpyDeviceToHost,
                                S->copy_stream) != cudaSuccess ||
                cudaStreamSynchronize(S->copy_stream) != cudaSuccess)
                st = QIEO_ERR_CUDA;
        }
        destroy_instance_nosync(q);
        std::lock_guard<std::mutex> lock(S->mu);
        R->inst = nullptr;
        if (st == QIEO_OK) S->alloc.release(R->off, R->bytes);   // a failed step keeps its memory
        R->status = st;
        R->state = st == QIEO_OK ? QIEO_SOLVE_DONE : QIEO_SOLVE_FAILED;
        R->t_done = server_now(S);
        if (st == QIEO_OK) S->n_completed += 1;
    }
    S->spare_events.push_back(rec.done);
    S->cv_done.notify_all();
}

void server_loop(qieo_server *S)
{
    cudaSetDevice(S->device);
    for (;;) {
        std::vector<SolveRequest *> admit;
        {
            std::unique_lock<std::mutex> lock(S->mu);
            while (!S->queue.empty() &&
                   (int64_t)(S->active.size() + admit.size()) < (int64_t)S->cfg.max_active) {
                SolveRequest *R = S->queue.front();
                size_t off = 0;
                if (!S->alloc.alloc(R->bytes, &off)) break;
                R->off = off;
                S->queue.pop_front();
                admit.push_back(R);
            }
            if (admit.empty() && S->active.empty() && S->inflight.empty()) {
                if (S->stop) break;
                S->cv_work.wait(lock);
                continue;
            }
        }
        for (SolveRequest *R : admit) {
            qieo_params pa = R->params;
            pa.stream = S->stream;
            pa.flags &= QIEO_FLAG_CONVERGE;
            pa.elite_on_host = 0;
            Placement pl{S->arena + R->off, R->bytes, R->gens};
            qieo_instance *q = nullptr;
            const qieo_status st = create_instance_impl(&R->prob, &pa, &pl, false, &q);
            std::lock_guard<std::mutex> lock(S->mu);
            R->t_admit = server_now(S);
            if (st == QIEO_OK) {
                R->inst = q;
                R->remaining = R->gens;
                R->state = QIEO_SOLVE_RUNNING;
                S->active.push_back(R);
                S->n_admitted += 1;
                S->n_launches += 1;   // the instance's generation-0 initialisation
                S->max_active_seen = std::max(S->max_active_seen, (int32_t)S->active.size());
            } else {
                S->alloc.release(R->off, R->bytes);
                R->status = st;
                R->state = QIEO_SOLVE_FAILED;
                R->t_done = R->t_admit;
                S->cv_done.notify_all();
            }
        }
        if (!S->active.empty() && S->inflight.size() < 2) {
            int32_t G = S->cfg.gens_per_step;
            std::vector<qieo_instance *> members;
            for (SolveRequest *R : S->active) {
                G = std::min(G, R->remaining);
                members.push_back(R->inst);
            }
            StepRecord rec;
            std::vector<qieo_instance *> watch;
            for (SolveRequest *R : S->active)
                if (R->params.flags & QIEO_FLAG_CONVERGE) {
                    rec.watched.push_back(R);
                    watch.push_back(R->inst);
                }
            int64_t launched = 0;
            qieo_status st = enqueue_server_step(S, members, G, &launched, watch, &rec.stop_host);
            if (st == QIEO_OK) {
                if (S->spare_events.empty()) {
                    cudaEvent_t ev = nullptr;
                    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) st = QIEO_ERR_CUDA;
                    S->spare_events.push_back(ev);
                }
            }
            if (st == QIEO_OK) {
                rec.done = S->spare_events.back();
                S->spare_events.pop_back();
                if (cudaEventRecord(rec.done, S->stream) != cudaSuccess) st = QIEO_ERR_CUDA;
            }
            std::lock_guard<std::mutex> lock(S->mu);
            std::vector<SolveRequest *> still;
            for (SolveRequest *R : S->active) {
                if (st != QIEO_OK) {
                    R->status = st;
                    R->state = QIEO_SOLVE_FAILED;
                    R->t_done = server_now(S);
                    continue;
                }
                R->remaining -= G;
                R->inst->t += G;
                if (R->remaining == 0) rec.finishing.push_back(R);
                else still.push_back(R);
            }
            S->active.swap(still);
            S->n_launches += launched;
            if (st == QIEO_OK) {
                S->n_steps += 1;
                S->inflight.push_back(rec);
            } else {
                S->cv_done.notify_all();
            }
        } else if (!S->inflight.empty()) {
            retire_oldest_step(S);
        }
    }
}

}  // namespace

extern "C" {

qieo_status qieo_server_create(const qieo_server_config *config, qieo_server **out)
{
    if (out) *out = nullptr;
    if (!out) return fail(QIEO_ERR_INVALID, "out is NULL");
    qieo_server_config cfg{};
    if (config) cfg = *config;
    if (cfg.memory_bytes < 0 || cfg.max_active < 0 || cfg.gens_per_step < 0)
        return fail(QIEO_ERR_INVALID, "negative server configuration");
    if (cfg.max_active == 0) cfg.max_active = 1024;
    if (cfg.gens_per_step == 0) cfg.gens_per_step = 25;
    qieo_server *S = new (std::nothrow) qieo_server();
    if (!S) return fail(QIEO_ERR_OOM, "host allocation failed");
    S->t0 = std::chrono::steady_clock::now();
    auto bail = [&](qieo_status st) {
        qieo_server_destroy(S);
        return st;
    };
    cudaError_t ce = cudaGetDevice(&S->device);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&S->sm_count, cudaDevAttrMultiProcessorCount, S->device);
    if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&S->copy_stream, cudaStreamNonBlocking);
    if (ce != cudaSuccess) return bail(fail(QIEO_ERR_CUDA, "server setup: %s", cudaGetErrorString(ce)));
    if (cfg.memory_bytes == 0) {
        size_t free_b = 0, total_b = 0;
        ce = cudaMemGetInfo(&free_b, &total_b);
        if (ce != cudaSuccess) return bail(fail(QIEO_ERR_CUDA, "cudaMemGetInfo: %s", cudaGetErrorString(ce)));
        cfg.memory_bytes = (int64_t)(free_b / 2);
    }
    S->cfg = cfg;
    ce = cudaMalloc(&S->arena, (size_t)cfg.memory_bytes);
    if (ce != cudaSuccess)
        return bail(fail(QIEO_ERR_OOM, "arena of %lld bytes: %s", (long long)cfg.memory_bytes, cudaGetErrorString(ce)));
    S->alloc.init((size_t)cfg.memory_bytes);
    for (int r = 0; r < 2; ++r) {
        ce = cudaMalloc(&S->wl_dev[r], kWorkListBytes);
        if (ce == cudaSuccess) ce = cudaMallocHost(&S->wl_host[r], kWorkListBytes);
        if (ce != cudaSuccess) return bail(fail(QIEO_ERR_OOM, "work lists: %s", cudaGetErrorString(ce)));
    }
    for (int narrow = 0; narrow < 2; ++narrow) {
        const size_t smem_max = qieo::kRingBytes + (size_t)qieo::kMaxSegRows * (narrow ? 8 : 16);
        for (int rule = 0; rule < 2; ++rule)
            for (int cip = 0; cip < 2; ++cip) {
                ce = cudaFuncSetAttribute(reinterpret_cast<const void *>(batch_kernel_of(narrow, rule, cip)),
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
                if (ce != cudaSuccess) return bail(fail(QIEO_ERR_CUDA, "kernel attribute: %s", cudaGetErrorString(ce)));
            }
        int bps = 0;
        ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &bps, reinterpret_cast<const void *>(batch_kernel_of(narrow, 0, true)), qieo::kThreads, smem_max);
        if (ce != cudaSuccess) return bail(fail(QIEO_ERR_CUDA, "occupancy: %s", cudaGetErrorString(ce)));
        S->bps[narrow] = std::max(1, bps);
    }
    S->worker = std::thread(server_loop, S);
    *out = S;
    return QIEO_OK;
}

qieo_status qieo_server_submit(qieo_server *S, const qieo_problem *pr, const qieo_params *pa,
                               int32_t generations, int64_t *id_out)
{
    if (!S || !pr || !pa || !id_out) return fail(QIEO_ERR_INVALID, "NULL argument");
    if (generations < 1) return fail(QIEO_ERR_INVALID, "generations must be >= 1");
    if (pr->ng < 1 || !pr->weights || !pr->values || pa->np < 1 || pr->capacity < 0 ||
        pa->dtheta_den < 4 || pa->dtheta_den > kMaxD || pa->dtheta_den % 4 != 0 ||
        pa->penalty_lambda < 1 || (pa->rotate_rule != 0 && pa->rotate_rule != 1))
        return fail(QIEO_ERR_INVALID, "invalid problem or params");
    for (int32_t j = 0; j < pr->ng; ++j)
        if (pr->weights[j] < 0) return fail(QIEO_ERR_INVALID, "weight %d is negative", j);
    size_t off[kParts];
    const size_t bytes = instance_layout(pr->ng, pa->np, pa->dtheta_den, generations, off);
    if (bytes > S->alloc.total())
        return fail(QIEO_ERR_OOM, "solve needs %zu bytes of device memory; the server arena holds %zu",
                    bytes, S->alloc.total());
    std::unique_ptr<SolveRequest> R(new (std::nothrow) SolveRequest());
    if (!R) return fail(QIEO_ERR_OOM, "host allocation failed");
    R->w.assign(pr->weights, pr->weights + pr->ng);
    R->v.assign(pr->values, pr->values + pr->ng);
    R->prob = *pr;
    R->prob.weights = R->w.data();
    R->prob.values = R->v.data();
    R->params = *pa;
    R->gens = generations;
    R->bytes = bytes;
    std::lock_guard<std::mutex> lock(S->mu);
    if (S->stop) return fail(QIEO_ERR_INVALID, "server is stopping");
    R->id = S->next_id++;
    R->t_submit = server_now(S);
    S->n_submitted += 1;
    *id_out = R->id;
    S->queue.push_back(R.get());
    S->all[R->id] = std::move(R);
    S->cv_work.notify_one();
    return QIEO_OK;
}

qieo_status qieo_server_poll(qieo_server *S, int64_t id, int32_t wait_ms, uint8_t *bits_out,
                             qieo_solve_result *res)
{
    if (!S || !res) return fail(QIEO_ERR_INVALID, "NULL argument");
    std::unique_lock<std::mutex> lock(S->mu);
    auto it = S->all.find(id);
    if (it == S->all.end()) return fail(QIEO_ERR_INVALID, "unknown request %lld", (long long)id);
    SolveRequest *R = it->second.get();
    if (wait_ms > 0)
        S->cv_done.wait_for(lock, std::chrono::milliseconds(wait_ms),
                            [&] { return R->state >= QIEO_SOLVE_DONE; });
    res->state = R->state;
    res->status = R->status;
    res->fitness = R->best[0];
    res->generation = (int32_t)R->best[1];
    res->chromosome = (int32_t)R->best[2];
    res->submit_s = R->t_submit;
    res->admit_s = R->t_admit;
    res->done_s = R->t_done;
    res->generations_run = R->gens_run;
    res->converged = R->converged;
    if (bits_out && R->state == QIEO_SOLVE_DONE) unpack_row(R->best_row.data(), R->prob.ng, bits_out);
    return QIEO_OK;
}

qieo_status qieo_server_get_stats(qieo_server *S, qieo_server_stats *out)
{
    if (!S || !out) return fail(QIEO_ERR_INVALID, "server and out must be non-NULL");
    std::lock_guard<std::mutex> lock(S->mu);
    out->submitted = S->n_submitted;
    out->admitted = S->n_admitted;
    out->completed = S->n_completed;
    out->steps = S->n_steps;
    out->kernel_launches = S->n_launches;
    out->queued = (int32_t)S->queue.size();
    out->active = (int32_t)S->active.size();
    out->max_active = S->max_active_seen;
    out->reserved = 0;
    return QIEO_OK;
}

qieo_status qieo_server_cancel(qieo_server *S, int64_t id)
{
    if (!S) return fail(QIEO_ERR_INVALID, "server is NULL");
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->all.find(id);
    if (it == S->all.end()) return fail(QIEO_ERR_INVALID, "unknown request %lld", (long long)id);
    SolveRequest *R = it->second.get();
    if (R->state != QIEO_SOLVE_QUEUED) return fail(QIEO_ERR_BUSY, "request %lld is no longer queued", (long long)id);
    S->queue.erase(std::find(S->queue.begin(), S->queue.end(), R));
    R->state = QIEO_SOLVE_CANCELLED;
    R->t_done = server_now(S);
    S->cv_done.notify_all();
    return QIEO_OK;
}

qieo_status qieo_server_destroy(qieo_server *S)
{
    if (!S) return QIEO_OK;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
        for (SolveRequest *R : S->queue) {
            R->state = QIEO_SOLVE_CANCELLED;
            R->t_done = server_now(S);
        }
        S->queue.clear();
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    cudaSetDevice(S->device);
    if (S->stream) cudaStreamSynchronize(S->stream);
    for (cudaEvent_t ev : S->spare_events) cudaEventDestroy(ev);
    for (int r = 0; r < 2; ++r) {
        if (S->wl_dev[r]) cudaFree(S->wl_dev[r]);
        if (S->wl_host[r]) cudaFreeHost(S->wl_host[r]);
    }
    if (S->arena) cudaFree(S->arena);
    if (S->stream) cudaStreamDestroy(S->stream);
    if (S->copy_stream) cudaStreamDestroy(S->copy_stream);
    delete S;
    return QIEO_OK;
}

qieo_status qieo_philox(const uint32_t *ctr_key, uint32_t *out, int32_t n)
{
    if (n < 0 || (n > 0 && (!ctr_key || !out))) return fail(QIEO_ERR_INVALID, "bad arguments");
    if (n == 0) return QIEO_OK;
    uint32_t *d_in = nullptr, *d_out = nullptr;
    CUDA_TRY(cudaMalloc(&d_in, (size_t)n * 6 * 4));
    cudaError_t ce = cudaMalloc(&d_out, (size_t)n * 4 * 4);
    if (ce == cudaSuccess) ce = cudaMemcpy(d_in, ctr_key, (size_t)n * 6 * 4, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) {
        qieo::philox_kernel<<<(n + 255) / 256, 256>>>(d_in, d_out, n);
        ce = cudaGetLastError();
    }
    if (ce == cudaSuccess) ce = cudaMemcpy(out, d_out, (size_t)n * 4 * 4, cudaMemcpyDeviceToHost);
    cudaFree(d_in);
    if (d_out) cudaFree(d_out);
    if (ce != cudaSuccess) return fail(QIEO_ERR_CUDA, "philox: %s", cudaGetErrorString(ce));
    return QIEO_OK;
}

}  // extern "C"
