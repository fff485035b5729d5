// qieo_kernels.cuh -- device code of the GB300 QIEO library.
//
// One generation (Sec. III-B, Fig. 1 of arxiv 2609.30862) is one fused pass over the qubit
// grid:
//   CIP(t-1)  rotate every qubit one step toward the previous elite's allele,
//   QIP(t)    observe every qubit against a Philox draw,
//   FE(t)     eq. (1) weight/value sums per chromosome (segmented reduction over genes),
//   DE(t)     the block that completes a chromosome's sums evaluates eq. (1) and folds
//             (fitness, -index) into one 64-bit atomic maximum; the last block to finish
//             the generation turns that maximum into the elite and the records.
// The CIP of generation t is applied at the top of generation t+1 because the elite is a
// grid-wide result, and once more after the last generation of a run.
//
// Two drivers of the same generation body:
//   run_kernel         one cooperative launch per run: all generations, a bounded grid
//                      barrier between them, and the final CIP (default path);
//   generation_kernel  one launch per generation (host DetermineElite variant, and runs
//                      that cannot be launched cooperatively), with cip_kernel at the end.
//
// Data layout in device memory (row c = chromosome c, gene-fastest, Sec. V-D):
//   state  uint16 4n, n = k + K in [0, 2K] (scaled by 4 so that it is the byte offset of
//          T[n] in the shared threshold table); rows padded to 8 genes; one uint4
//          ("vector") = 8 genes.
//   xbits  [2][np][xstride]: alleles of generation t in plane t & 1; bit i of byte v is
//          gene 8v + i; rows padded to 16 bytes.
//   items  narrow: uint32 (v << 16 | w) per gene; wide: int32 w[], int32 v[].
//   acc    narrow: uint64 (count << 52 | SV << 26 | SW) per row; wide: int64 SW, SV per row
//          plus a uint32 count per row.
//
// Work split: a generation is ntile * np tile-rows (tile = lanes*warps vectors of one row).
// Each block of the grid owns a contiguous, equal share of them in tile-major order, so it
// reloads items only at a tile change and keeps the same share in every generation.
#pragma once

#include <type_traits>

#include <cstdint>
#include <cuda_runtime.h>

#include "qieo_device.cuh"

namespace qieo {

constexpr int kThreads = 256;
constexpr int kMaxSegRows = 1536;          // tile-rows summed in shared memory at once
constexpr int kMaxK = 1000;                // D <= 4000
constexpr int kMaxThr = 2 * kMaxK + 1;

// ---------------------------------------------------------------------------------------
// Small PTX helpers: programmatic dependent launch, acquire/release accesses, the clock.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void grid_dependency_wait()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

__device__ __forceinline__ void allow_dependent_launch()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ unsigned int atom_add_acq_rel(unsigned int *p, unsigned int v)
{
    unsigned int old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;"
                 : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int32_t ld_acquire(const int32_t *p)
{
    int32_t v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int32_t *p, int32_t v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Elite key: larger fitness wins, then the lower chromosome index.
constexpr int64_t kKeyBias = (int64_t)1 << 39;

__device__ __forceinline__ unsigned long long elite_key(int64_t f, int32_t c)
{
    return ((unsigned long long)(f + kKeyBias) << 24) | (unsigned long long)(0xffffffu - (uint32_t)c);
}

// Error bits reported through GenParams::error.
constexpr int32_t kErrBarrierTimeout = 1;
constexpr int32_t kErrEliteRange = 2;   // a generation closed with no chromosome finished

struct GenParams {
    uint4 *state;                 // [np][svec] scaled angle indices
    uint8_t *xbits;               // [2][np][xstride]
    const uint4 *items_narrow;    // [2 svec] packed (v << 16 | w), 4 genes per uint4, then
                                  // [svec] byte vectors (w0 w2 w1 w3, w4 w6 w5 w7, same for v)
    const int4 *w4;               // wide: [2 svec] weights
    const int4 *v4;               // wide: [2 svec] values
    unsigned long long *acc;      // narrow [np]; wide [2 np]
    unsigned int *cnt;            // wide: [np]
    int64_t *fitness;             // [np] of the last generation
    unsigned long long *keys;     // [3] elite key of generation t in slot t % 3
    int32_t *elite_idx;           // [1] elite of the last completed generation
    int32_t *hist_e;              // [capacity] elite index per generation
    int64_t *hist_f;              // [capacity] elite fitness per generation
    int64_t *best;                // [3] fitness, generation (-1 none), chromosome
    uint8_t *best_row;            // [xstride]
    int32_t *gen;                 // number of the generation to run next
    unsigned int *ticket;         // blocks finished in this generation
    int32_t *bar_gen;             // grid barrier: generations released so far
    int32_t *error;               // kErr* bits
    int32_t *conv;                // [4] convergence test: run length of equal elite
                                  // fitness ending at generation t in conv[t & 1], the
                                  // stop state (kRunning, kStopPending: the final CIP is
                                  // still due, kStopped) in conv[2], and in conv[3] the
                                  // generation that met the test
    const uint32_t *thr;          // [2K+1] low 32 bits of T[n] (T[2K] = 2^32 -> 0)
    int64_t capacity, lambda;
    int64_t units;                // ntile * np tile-rows
    size_t xplane;                // np * xstride
    uint64_t wait_ns;             // bound of one grid-barrier wait
    int32_t np, svec, xstride, K, ntile;
    int32_t lanes, warps, seg_rows_max, key_mode;
    int32_t apply_cip, do_de;
    int32_t ring;                 // 1: state streamed through the per-thread cp.async ring
    int32_t converge;             // 1: stop once the elite fitness is stable (kConvergeWindow)
    int32_t g;                    // generation of this launch within its run (deferred
                                  // close: t = *gen + g; otherwise 0 and t = *gen)
    int32_t deferred;             // 1: deferred close (see generation_kernel)
    int32_t state8;               // 1: angle indices stored as bytes (8 B per 8 genes)
    const int4 *segq;             // segment queue (tile, first row, rows, 0) of the deferred
                                  // forms, in order of decreasing size; nsegs = 0: none
    unsigned int *qctr;           // [3] next queue index of generation t in slot t % 3
    int32_t nsegs;
    int32_t row0;                 // chromosome index of row 0 in the draws' counters (a row
                                  // block of a population sharded by rows; 0 otherwise)
    unsigned long long *gen_ns;   // resident form: device clock (ns) at the start of each
                                  // generation of the run and at its end, or NULL
    uint32_t *fword;              // [np][fstride / 32] fixed-vector words of the stored state
                                  // (one bit per vector, see below), or NULL when the instance
                                  // keeps none
    unsigned long long *fcnt;     // [7] vectors whose F is nonzero after generation t, in
                                  // slot t % 3 (an estimate while the words are not kept);
                                  // [3]: 1 once the words are kept; [4 + t % 3]: vectors
                                  // that did not draw in generation t
    unsigned long long *hist_d;   // [capacity] vectors that did not draw, per generation
                                  // (copied from fcnt once the generation is complete), or
                                  // NULL
    unsigned long long *fprev;    // [np] packed row totals (SV << 26 | SW) of the last
                                  // generation, kept by the kernel that keeps F
    const uint32_t *ftile;        // [2 ntile] sums of the weights and of the values of each
                                  // tile's genes (the bias of a sparse generation's changes)
    int64_t fsum_w, fsum_v;       // sums of all weights and of all values
    int32_t fstride;              // vectors of a row of F: ntile * 256 (fstride / 32 words)
    unsigned long long sparse_min;   // a generation takes the sparse form when at least
                                     // this many vectors were fixed after the one before
    unsigned long long f_on_min;     // the words are kept from the first generation after
                                     // one whose estimate of fixed vectors reached this
    uint32_t rk0[10], rk1[10];    // Philox round keys of (seed, instance)
};

// Convergence stop (Sec. IV, Workload): the run stops once the elite fitness has been the
// same for kConvergeWindow consecutive generations (integer fitness: "within 1e-6 of the
// mean" is equality). The generation that meets it still gets its CIP (Fig. 1 order): the
// next launch of the instance applies it alone and marks the instance stopped.
constexpr int32_t kConvergeWindow = 20;
constexpr int32_t kRunning = 0, kStopPending = 1, kStopped = 2;

__device__ __forceinline__ int32_t stop_state(const GenParams &p)
{
    return p.converge ? *(volatile const int32_t *)(p.conv + 2) : kRunning;
}

__device__ __forceinline__ unsigned long long *key_slot(const GenParams &p, int32_t t)
{
    return p.keys + (t % 3);
}

// Eq. (1) of a finished row; records the fitness and offers the row to the elite key.
__device__ __forceinline__ void finish_row(const GenParams &p, int32_t c, int64_t sw, int64_t sv,
                                           int32_t t)
{
    const int64_t f = sw <= p.capacity ? sv : -p.lambda * (sw - p.capacity);
    p.fitness[c] = f;
    if (p.key_mode) atomicMax(key_slot(p, t), elite_key(f, c));
}

// Adds one block's sums of a tile-row to the row; the block that adds the last of the
// ntile contributions evaluates the row.
template <bool kNarrow>
__device__ __forceinline__ void combine_row(const GenParams &p, int32_t c, uint64_t sw, uint64_t sv,
                                            int32_t t)
{
    if (kNarrow) {
        const unsigned long long add = (1ull << 52) | (sv << 26) | sw;
        const unsigned long long old = atomicAdd(p.acc + c, add);
        if ((int32_t)(old >> 52) == p.ntile - 1) {
            const unsigned long long full = old + add;
            p.acc[c] = 0ull;
            finish_row(p, c, (int64_t)(full & 0x3ffffffull), (int64_t)((full >> 26) & 0x3ffffffull), t);
        }
    } else {
        atomicAdd(p.acc + 2 * (size_t)c, (unsigned long long)sw);
        atomicAdd(p.acc + 2 * (size_t)c + 1, (unsigned long long)sv);
        if ((int32_t)atom_add_acq_rel(p.cnt + c, 1u) == p.ntile - 1) {
            const int64_t w = (int64_t)ld_relaxed(p.acc + 2 * (size_t)c);
            const int64_t v = (int64_t)ld_relaxed(p.acc + 2 * (size_t)c + 1);
            p.acc[2 * (size_t)c] = 0ull;
            p.acc[2 * (size_t)c + 1] = 0ull;
            p.cnt[c] = 0u;
            finish_row(p, c, w, v, t);
        }
    }
}

// Closes generation t (one block, all threads): elite from the key (or a lowest-index
// argmax over the fitness array when fitness values do not fit the key), records.
__device__ void close_generation(const GenParams &p, int32_t t)
{
    __shared__ int64_t s_f[kThreads / 32];
    __shared__ int32_t s_c[kThreads / 32];
    __shared__ int32_t s_e;
    __shared__ int32_t s_improved;
    const int tid = threadIdx.x;
    int64_t bf = INT64_MIN;
    int32_t bc = 0x7fffffff;
    // the previous best record, loaded together with the elite key (one round trip)
    const int64_t best_f = tid == 0 ? __ldcg(p.best) : 0, best_g = tid == 0 ? __ldcg(p.best + 1) : 0;
    if (p.key_mode) {
        if (tid == 0) {
            const unsigned long long k = __ldcg(key_slot(p, t));
            bc = (int32_t)(0xffffffu - (uint32_t)(k & 0xffffffull));
            bf = (int64_t)(k >> 24) - kKeyBias;
            *key_slot(p, t) = 0ull;
        }
    } else {
        for (int c = tid; c < p.np; c += kThreads) {
            const int64_t f = __ldcg(p.fitness + c);
            if (f > bf) {   // c grows within a thread: the first maximum is kept
                bf = f;
                bc = c;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const int64_t of = __shfl_xor_sync(0xffffffffu, bf, o);
            const int32_t oc = __shfl_xor_sync(0xffffffffu, bc, o);
            if (of > bf || (of == bf && oc < bc)) {
                bf = of;
                bc = oc;
            }
        }
        if ((tid & 31) == 0) {
            s_f[tid >> 5] = bf;
            s_c[tid >> 5] = bc;
        }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < kThreads / 32; ++w) {
                if (s_f[w] > bf || (s_f[w] == bf && s_c[w] < bc)) {
                    bf = s_f[w];
                    bc = s_c[w];
                }
            }
        }
    }
    if (tid == 0) {
        // Every row finishes in every generation, so the elite lies in [0, np); anything
        // else is recorded as an internal error and replaced by row 0 so that no later
        // access leaves the population.
        if (bc < 0 || bc >= p.np) {
            atomicOr(p.error, kErrEliteRange);
            bc = 0;
        }
        if (p.converge) {
            const int32_t prev = t > 0 ? p.conv[(t - 1) & 1] : 0;
            const int32_t run = (prev > 0 && bf == p.hist_f[t - 1]) ? prev + 1 : 1;
            p.conv[t & 1] = run;
            if (run >= kConvergeWindow) {
                p.conv[3] = t;
                p.conv[2] = kStopPending;
            }
        }
        p.hist_e[t] = bc;
        p.hist_f[t] = bf;
        *p.elite_idx = bc;
        const int improved = (best_g < 0 || bf > best_f) ? 1 : 0;
        if (improved) {
            p.best[0] = bf;
            p.best[1] = t;
            p.best[2] = bc;
        }
        s_e = bc;
        s_improved = improved;
    }
    __syncthreads();
    if (s_improved) {
        const uint4 *src = reinterpret_cast<const uint4 *>(
            p.xbits + (size_t)(t & 1) * p.xplane + (size_t)s_e * p.xstride);
        uint4 *dst = reinterpret_cast<uint4 *>(p.best_row);
        for (int i = tid; i < p.xstride / 16; i += kThreads) dst[i] = __ldcg(src + i);
    }
    __syncthreads();
}

// Per-block constants of the work split.
struct BlockShare {
    int tile_vecs, rows_per_pass, r_sub, v_in, lanes;
    bool leader;                  // first lane of its row segment
    int64_t u_begin, u_end;       // tile-rows [u_begin, u_end) of this block
};

// Thread geometry of a tile of lanes x warps vectors in a block of kThreads threads.
// (lanes and warps are powers of two, so the split is shifts and masks)
__device__ __forceinline__ BlockShare tile_geometry(int lanes, int warps)
{
    BlockShare b;
    b.lanes = lanes;
    b.tile_vecs = lanes * warps;
    const int sh = __ffs(b.tile_vecs) - 1;
    b.rows_per_pass = kThreads >> sh;
    b.r_sub = threadIdx.x >> sh;
    b.v_in = threadIdx.x & (b.tile_vecs - 1);
    b.leader = (threadIdx.x & (lanes - 1)) == 0;
    b.u_begin = 0;
    b.u_end = 0;
    return b;
}

// Tile-rows [u_begin, u_end) of this block: an equal split of the ntile * np tile-rows, in
// 32-bit arithmetic whenever the products fit (a 64-bit division is a long software routine).
__device__ __forceinline__ BlockShare block_share(const GenParams &p)
{
    BlockShare b = tile_geometry(p.lanes, p.warps);
    const uint64_t units = (uint64_t)p.units;
    if (units * gridDim.x <= 0xffffffffull) {
        const uint32_t u = (uint32_t)units;
        b.u_begin = (int64_t)((blockIdx.x * u) / gridDim.x);
        b.u_end = (int64_t)(((blockIdx.x + 1u) * u) / gridDim.x);
    } else {
        b.u_begin = (int64_t)blockIdx.x * p.units / gridDim.x;
        b.u_end = (int64_t)(blockIdx.x + 1) * p.units / gridDim.x;
    }
    return b;
}

__device__ __forceinline__ void load_thresholds(const GenParams &p, uint32_t *s_thr)
{
    for (int i = threadIdx.x; i < 2 * p.K + 1; i += kThreads) s_thr[i] = p.thr[i];
}

// Sum over the lanes of a row segment (lanes lanes, a power of two).
template <bool kNarrow>
__device__ __forceinline__ void segment_sum(int lanes, uint32_t &accn, int64_t &acw, int64_t &acv)
{
    if (kNarrow) {
        if (lanes == 32) {
            accn = __reduce_add_sync(0xffffffffu, accn);
        } else {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                if (o < lanes) accn += __shfl_xor_sync(0xffffffffu, accn, o);
        }
    } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            if (o < lanes) {
                acw += __shfl_xor_sync(0xffffffffu, acw, o);
                acv += __shfl_xor_sync(0xffffffffu, acv, o);
            }
        }
    }
}

// Per-segment constants of one thread: its vector of a tile, the 8 items of that vector
// and the elite alleles of the previous generation for it.
//
// Narrow items are kept twice: packed (v << 16 | w) per gene in registers, added under the
// allele predicates of a drawn pass; and as four byte vectors w4a = (w0, w2, w1, w3),
// w4b = (w4, w6, w5, w7) and the same for v in the thread's slot of s_item_bytes, where a
// fixed-allele pass forms its sums as byte dot products (dp4a) with allele bytes built in
// the same order (see allele_nibble_hi).
struct SegCtx {
    uint32_t wv[8];               // narrow items (v << 16 | w)
    int32_t wi[8], vi[8];         // wide items
    uint32_t e8;                  // elite alleles of the previous generation (8 genes)
    uint32_t ctr0;                // Philox counter word 0 of the first 4 genes
    int vec;
    bool active;                  // vec < svec
};

__shared__ uint4 s_item_bytes[kThreads];   // per thread: w4a, w4b, v4a, v4b
// Rule R1 moves every qubit toward the elite's allele, so the CIP deltas of a vector depend
// only on the elite's 8 alleles: kernels built with kSegDelta form them once per segment
// (four delta_pair words, as signed steps for rotate_pair_signed) into this per-thread
// slot, and a pass reads them with one 16-byte shared load instead of forming them (see
// ring_segment for where it pays).
__shared__ uint4 s_delta[kThreads];

// The elite alleles of the thread's vector; kSegDelta: also the rule R1 delta words of the
// segment (s_delta).
template <bool kCip, bool kSegDelta = false>
__device__ __forceinline__ void seg_elite(SegCtx &g, const uint8_t *elite_row)
{
    g.e8 = (kCip && g.active) ? (uint32_t)__ldcg(elite_row + g.vec) : 0u;
    if (kCip && kSegDelta)   // read back by this thread only (rule R1 passes)
        s_delta[threadIdx.x] = make_uint4(signed_step(delta_pair(g.e8 & 3u, 3u)),
                                          signed_step(delta_pair((g.e8 >> 2) & 3u, 3u)),
                                          signed_step(delta_pair((g.e8 >> 4) & 3u, 3u)),
                                          signed_step(delta_pair((g.e8 >> 6) & 3u, 3u)));
}

// The thread's vector of a tile and its 8 items (registers, and the byte vectors in the
// thread's slot of s_item_bytes).
template <bool kNarrow>
__device__ __forceinline__ void seg_items(const GenParams &p, SegCtx &g, int tile, int v_in, int tile_vecs)
{
    g.vec = tile * tile_vecs + v_in;
    g.active = g.vec < p.svec;
    if (kNarrow) {
        uint4 a = make_uint4(0, 0, 0, 0), c = a, d = a;
        if (g.active) {
            a = __ldg(p.items_narrow + 2 * (size_t)g.vec);
            c = __ldg(p.items_narrow + 2 * (size_t)g.vec + 1);
            d = __ldg(p.items_narrow + 2 * (size_t)p.svec + g.vec);
        }
        g.wv[0] = a.x; g.wv[1] = a.y; g.wv[2] = a.z; g.wv[3] = a.w;
        g.wv[4] = c.x; g.wv[5] = c.y; g.wv[6] = c.z; g.wv[7] = c.w;
        s_item_bytes[threadIdx.x] = d;   // read back by this thread only
    } else {
        int4 a = make_int4(0, 0, 0, 0), c = a, d = a, e = a;
        if (g.active) {
            a = __ldg(p.w4 + 2 * (size_t)g.vec);
            c = __ldg(p.w4 + 2 * (size_t)g.vec + 1);
            d = __ldg(p.v4 + 2 * (size_t)g.vec);
            e = __ldg(p.v4 + 2 * (size_t)g.vec + 1);
        }
        g.wi[0] = a.x; g.wi[1] = a.y; g.wi[2] = a.z; g.wi[3] = a.w;
        g.wi[4] = c.x; g.wi[5] = c.y; g.wi[6] = c.z; g.wi[7] = c.w;
        g.vi[0] = d.x; g.vi[1] = d.y; g.vi[2] = d.z; g.vi[3] = d.w;
        g.vi[4] = e.x; g.vi[5] = e.y; g.vi[6] = e.z; g.vi[7] = e.w;
    }
    g.ctr0 = 2u * (uint32_t)g.vec;
}

template <bool kNarrow, bool kCip, bool kSegDelta = false>
__device__ __forceinline__ void seg_setup(const GenParams &p, SegCtx &g, int tile, int v_in,
                                          int tile_vecs, const uint8_t *elite_row)
{
    seg_items<kNarrow>(p, g, tile, v_in, tile_vecs);
    seg_elite<kCip, kSegDelta>(g, elite_row);
}

// Philox key sources: the ten round keys of a single instance live in the kernel parameter
// block (each xor reads its key from the constant bank); a batch computes the schedule of
// the current instance's (block-uniform) key inline.
struct ParamKeys {
    const GenParams &p;
    __device__ __forceinline__ Draw4 operator()(uint32_t c0, uint32_t c1, uint32_t c2) const
    {
        return philox4x32_10_rk(c0, c1, c2, 0u, p.rk0, p.rk1);
    }
};

struct InlineKeys {
    uint32_t k0, k1;
    __device__ __forceinline__ Draw4 operator()(uint32_t c0, uint32_t c1, uint32_t c2) const
    {
        return philox4x32_10(c0, c1, c2, 0u, k0, k1);
    }
};

// Bytes (x0, x2, x1, x3), each 0 or 1 -> nibble (bit i = x_i). The terms shift byte 0 to
// bit 24, byte 1 to bit 26, byte 2 to bit 25 and byte 3 to bit 27; the other partial
// products fall below bit 20 or at bit 32 and above, again without carries.
__device__ __forceinline__ uint32_t allele_nibble_hi(uint32_t bytes)
{
    return bytes * 0x01040208u;   // the nibble is bits 24..27
}

// Packed narrow sums (sum v << 16 | sum w) of the 8 genes of a pass from allele bytes
// (x0, x2, x1, x3) and (x4, x6, x5, x7).
__device__ __forceinline__ uint32_t narrow_sums(uint32_t xa, uint32_t xb)
{
    const uint4 ib = s_item_bytes[threadIdx.x];
    const uint32_t sw = __dp4a(xa, ib.x, __dp4a(xb, ib.y, 0u));
    const uint32_t sv = __dp4a(xa, ib.z, __dp4a(xb, ib.w, 0u));
    return sw | (sv << 16);
}

// Fixed-vector words. F of a vector of the stored state is 1 when all eight of its qubits
// sit at theta = 0 or pi/2 (n = 0 or 2K: each allele is then the side of its bound whatever
// the draw), else 0; 0 is also always a safe value ("not known to be fixed"), so F may be
// cleared at any time. Instances that keep F store it row-major, one bit per vector, 32
// vectors to a 32-bit word, fstride / 32 words a row. A fixed vector's sides are its alleles
// of the generation that observed that state, so F and the previous allele plane together
// say whether a vector is stable.

// Alleles of four genes (bit i = gene i of the nibble) -> bytes (x0, x2, x1, x3), the order
// narrow_sums takes: the multiplier's terms 1, 2^15, 2^6, 2^21 move bit 0 to bit 0, bit 1 to
// 16, bit 2 to 8 and bit 3 to 24, and the sixteen partial products all land on different
// bits, so nothing carries.
__device__ __forceinline__ uint32_t allele_bytes(uint32_t nib)
{
    return (nib * 0x00208041u) & 0x01010101u;
}

// One vector of one row: CIP(t-1), QIP(t), the row's partial sums. Returns the new state
// and the packed or wide sums through accn / acw, acv (before the segment reduction).
//
// Fixed-allele pass: a qubit at theta = 0 or pi/2 (n = 0 or 2K, T = 0 or 2^32) yields the
// same allele for every draw, and CIP leaves it where it is when it already sits at the
// bound on the elite's side (or is not rotated). When that holds for every qubit of the
// pass in the whole warp, the alleles are the bits of the state itself, no Philox call is
// needed, and the state is unchanged (fixed = true: the caller skips its store). The test
// is skipped for 15 passes after it fails, which keeps its cost low while the population
// is still spread out. (An exponential backoff, 1, 3, 7 then 15 passes, measured slower:
// c3's saturated generations 186 vs 177 us, c2's spread ones 15.8 vs 14.9 us.)
//
// zor (when not NULL) receives the OR of the eight threshold words the pass compared
// against: 0 exactly when every qubit of the vector sits at theta = 0 or pi/2 after the
// rotation (T[0] = 0 and T[2K] = 2^32 have zero low words, every T[n] in between has not).
template <bool kNarrow, int kRule, bool kCip, class Keys, bool kSegDelta = false>
__device__ __forceinline__ uint4 qubit_pass(const GenParams &p, const Keys &keys, const SegCtx &g, uint4 s,
                                            uint32_t xo, int32_t c, int32_t t,
                                            const unsigned char *thr_bytes, bool &fixed,
                                            int &countdown, uint32_t &xbits, uint32_t &accn,
                                            int64_t &acw, int64_t &acv, uint32_t *zor = nullptr,
                                            uint32_t *nsat = nullptr, uint32_t *nskip = nullptr)
{
    const uint32_t off_top = (uint32_t)(8 * p.K);
    const uint32_t k8 = off_top * 0x00010001u;
    const uint32_t m8 = kRule == 1 ? (g.e8 ^ xo) : 0xffu;   // genes the rotation moves
    accn = 0u;
    acw = 0;
    acv = 0;
    fixed = false;

    if (countdown == 0) {
        // A half h in {0, 8K} is h == b * 8K with b its bit number bp (any set bit of 8K).
        const int bp = __ffs((int)off_top) - 1;
        const uint32_t b0 = (s.x >> bp) & 0x00010001u, b1 = (s.y >> bp) & 0x00010001u;
        const uint32_t b2 = (s.z >> bp) & 0x00010001u, b3 = (s.w >> bp) & 0x00010001u;
        const bool sat = s.x == b0 * off_top && s.y == b1 * off_top && s.z == b2 * off_top &&
                         s.w == b3 * off_top;
        // b0 holds gene 0 at bit 0 and gene 1 at bit 16, so xa = (x0, x2, x1, x3) as bytes
        const uint32_t xa = b0 | (b1 << 8), xb = b2 | (b3 << 8);
        const uint32_t xs = (allele_nibble_hi(xa) >> 24) | ((allele_nibble_hi(xb) >> 20) & 0xf0u);
        const bool ok = sat && (!kCip || ((g.e8 ^ xs) & m8) == 0u);
        if (nsat && sat && g.active) *nsat += 16u;
        if (__all_sync(0xffffffffu, ok)) {
            fixed = true;
            xbits = xs;
            if (zor) *zor = 0u;
            if (nskip && g.active) ++*nskip;
            if (kNarrow) {
                accn = narrow_sums(xa, xb);
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    if ((xs >> i) & 1u) {
                        acw += g.wi[i];
                        acv += g.vi[i];
                    }
                }
            }
            return s;
        }
        countdown = 15;
    } else {
        --countdown;
    }

    if (kCip) {
        if (kRule == 0 && kSegDelta) {  // R1: the segment's signed steps
            const uint4 d = s_delta[threadIdx.x];
            s.x = rotate_pair_signed(s.x, d.x, k8);
            s.y = rotate_pair_signed(s.y, d.y, k8);
            s.z = rotate_pair_signed(s.z, d.z, k8);
            s.w = rotate_pair_signed(s.w, d.w, k8);
        } else {
            s = rotate_vec(s, g.e8, m8, k8);
        }
    }
    const uint32_t sp[4] = {s.x, s.y, s.z, s.w};
    const Draw4 r0 = keys(g.ctr0, (uint32_t)c, (uint32_t)t);
    const Draw4 r1 = keys(g.ctr0 + 1u, (uint32_t)c, (uint32_t)t);
    const uint32_t u[8] = {r0.a, r0.b, r0.c, r0.d, r1.a, r1.b, r1.c, r1.d};
    xbits = 0u;
    uint32_t z = 0u;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const uint32_t off = (i & 1) ? (sp[i >> 1] >> 16) : (sp[i >> 1] & 0xffffu);
        const uint32_t thr = *reinterpret_cast<const uint32_t *>(thr_bytes + off);
        z |= thr;
        if ((u[i] < thr) || (off == off_top)) {
            xbits |= 1u << i;
            if (kNarrow) {
                accn += g.wv[i];
            } else {
                acw += g.wi[i];
                acv += g.vi[i];
            }
        }
    }
    if (zor) *zor = z;
    return s;
}

template <bool kNarrow>
__device__ __forceinline__ void add_row_sums(int lanes, bool leader, bool ok, int rr,
                                             uint32_t accn, int64_t acw, int64_t acv,
                                             uint32_t *s_acc32, unsigned long long *s_acc64)
{
    uint32_t a = accn;
    int64_t w = acw, v = acv;
    segment_sum<kNarrow>(lanes, a, w, v);
    if (ok && leader) {
        if (kNarrow) {
            atomicAdd(s_acc32 + 2 * rr, a & 0xffffu);
            atomicAdd(s_acc32 + 2 * rr + 1, a >> 16);
        } else {
            atomicAdd(s_acc64 + 2 * rr, (unsigned long long)w);
            atomicAdd(s_acc64 + 2 * rr + 1, (unsigned long long)v);
        }
    }
}

// The kernel that keeps F also keeps every row's totals (fprev): a dense generation adds
// the tile-rows' sums as combine_row<true> does and the block that finishes a row stores
// its totals; a sparse generation adds only the signed changes of the vectors it drew
// again, each tile-row's change biased by its tile's item sums so that the packed fields
// stay non-negative, and the block that finishes the row removes the biases (their total is
// the sum of all items) and adds the change to the totals of the generation before.
__device__ __forceinline__ void combine_row_keep(const GenParams &p, int32_t c, uint64_t sw, uint64_t sv,
                                                 int32_t t)
{
    const unsigned long long add = (1ull << 52) | (sv << 26) | sw;
    const unsigned long long old = atomicAdd(p.acc + c, add);
    if ((int32_t)(old >> 52) == p.ntile - 1) {
        const unsigned long long full = old + add;
        p.acc[c] = 0ull;
        p.fprev[c] = full & ((1ull << 52) - 1ull);
        finish_row(p, c, (int64_t)(full & 0x3ffffffull), (int64_t)((full >> 26) & 0x3ffffffull), t);
    }
}

__device__ __forceinline__ void combine_row_delta(const GenParams &p, int32_t c, int32_t dw, int32_t dv,
                                                  uint32_t bw, uint32_t bv, int32_t t)
{
    // dw + bw >= 0 (a tile-row's sum cannot drop by more than its tile's weights), and the
    // ntile biased changes add up to at most 2 fsum_w < 2^26, so the fields never carry
    const unsigned long long add = (1ull << 52) | ((unsigned long long)(uint32_t)(dv + (int32_t)bv) << 26) |
                                   (unsigned long long)(uint32_t)(dw + (int32_t)bw);
    const unsigned long long old = atomicAdd(p.acc + c, add);
    if ((int32_t)(old >> 52) == p.ntile - 1) {
        const unsigned long long full = old + add;
        p.acc[c] = 0ull;
        const unsigned long long prev = p.fprev[c];
        const int64_t SW = (int64_t)(prev & 0x3ffffffull) + (int64_t)(full & 0x3ffffffull) - p.fsum_w;
        const int64_t SV = (int64_t)((prev >> 26) & 0x3ffffffull) + (int64_t)((full >> 26) & 0x3ffffffull) - p.fsum_v;
        p.fprev[c] = ((unsigned long long)SV << 26) | (unsigned long long)SW;
        finish_row(p, c, SW, SV, t);
    }
}

// Adds the block's tile-row sums of a segment to the rows (one atomic per tile-row) and
// clears the shared accumulators. Called by the whole block. kMode 1: the packed sums
// with the row totals kept (combine_row_keep); kMode 2: signed 32-bit changes
// (combine_row_delta).
template <bool kNarrow, int kMode = 0>
__device__ __forceinline__ void flush_segment(const GenParams &p, int32_t t, int ra, int seg_rows,
                                              uint32_t *s_acc32, unsigned long long *s_acc64, int tile = 0)
{
    __syncthreads();
    const uint32_t bw = kMode == 2 ? __ldg(p.ftile + 2 * tile) : 0u;
    const uint32_t bv = kMode == 2 ? __ldg(p.ftile + 2 * tile + 1) : 0u;
    for (int i = threadIdx.x; i < seg_rows; i += kThreads) {
        if (kMode == 2) {
            combine_row_delta(p, ra + i, (int32_t)s_acc32[2 * i], (int32_t)s_acc32[2 * i + 1], bw, bv, t);
            s_acc32[2 * i] = 0u;
            s_acc32[2 * i + 1] = 0u;
        } else if (kMode == 1) {
            combine_row_keep(p, ra + i, s_acc32[2 * i], s_acc32[2 * i + 1], t);
            s_acc32[2 * i] = 0u;
            s_acc32[2 * i + 1] = 0u;
        } else if (kNarrow) {
            combine_row<true>(p, ra + i, s_acc32[2 * i], s_acc32[2 * i + 1], t);
            s_acc32[2 * i] = 0u;
            s_acc32[2 * i + 1] = 0u;
        } else {
            combine_row<false>(p, ra + i, s_acc64[2 * i], s_acc64[2 * i + 1], t);
            s_acc64[2 * i] = 0ull;
            s_acc64[2 * i + 1] = 0ull;
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------------------
// One generation over this block's share, register-prefetch form (any tile shape).
// Thread (r_sub, v_in) handles vector v_in of rows r_sub, r_sub + rows_per_pass, ... of
// each tile segment; its 8 items stay in registers for the whole segment, and the state of
// the next two rows is in flight while a row is computed. Row sums are reduced over the
// lanes of a segment in the warp, over the warps of a tile in shared memory, and over tiles
// by one atomic per tile-row.
// ---------------------------------------------------------------------------------------
template <bool kNarrow, int kRule, bool kCip>
__device__ __forceinline__ void generation_body(const GenParams &p, const BlockShare &b,
                                                int32_t t, int32_t e_prev,
                                                const uint32_t *s_thr, uint32_t *s_acc32,
                                                unsigned long long *s_acc64)
{
    const unsigned char *thr_bytes = reinterpret_cast<const unsigned char *>(s_thr);
    const uint8_t *x_prev = p.xbits + (size_t)((t + 1) & 1) * p.xplane;
    uint8_t *x_cur = p.xbits + (size_t)(t & 1) * p.xplane;
    const uint8_t *elite_row = x_prev + (size_t)e_prev * p.xstride;
    const int rpp = b.rows_per_pass;
    int countdown = 0;

    for (int i = threadIdx.x; i < 2 * p.seg_rows_max; i += kThreads) {
        if (kNarrow) s_acc32[i] = 0u;
        else s_acc64[i] = 0ull;
    }
    __syncthreads();

    for (int64_t u0 = b.u_begin; u0 < b.u_end;) {
        const int tile = (int)(u0 / p.np);
        const int ra = (int)(u0 - (int64_t)tile * p.np);
        const int seg_rows = (int)min(min((int64_t)(p.np - ra), b.u_end - u0), (int64_t)p.seg_rows_max);
        u0 += seg_rows;
        const int passes = (seg_rows + rpp - 1) / rpp;

        SegCtx g;
        seg_setup<kNarrow, kCip>(p, g, tile, b.v_in, b.tile_vecs, elite_row);
        const size_t row0 = (size_t)ra + b.r_sub;
        uint4 *sptr = p.state + row0 * p.svec + g.vec;
        const size_t sstep = (size_t)rpp * p.svec;
        uint8_t *xptr = x_cur + row0 * p.xstride + g.vec;
        const uint8_t *xoptr = x_prev + row0 * p.xstride + g.vec;
        const size_t xstep = (size_t)rpp * p.xstride;

        auto row_ok = [&](int pass) { return pass * rpp + b.r_sub < seg_rows; };
        auto load_state = [&](int pass) -> uint4 {
            uint4 v = make_uint4(0, 0, 0, 0);
            if (g.active && row_ok(pass)) v = sptr[(size_t)pass * sstep];
            return v;
        };
        auto load_xold = [&](int pass) -> uint32_t {
            if (kRule != 1 || !kCip) return 0u;
            if (!(g.active && row_ok(pass))) return 0u;
            return (uint32_t)xoptr[(size_t)pass * xstep];
        };
        auto process = [&](uint4 sv, uint32_t xo, int pass) {
            const int rr = pass * rpp + b.r_sub;
            const bool ok = rr < seg_rows;
            uint32_t xbits, accn;
            int64_t acw, acv;
            bool fixed;
            sv = qubit_pass<kNarrow, kRule, kCip>(p, ParamKeys{p}, g, sv, xo, ra + p.row0 + rr, t, thr_bytes,
                                                  fixed, countdown, xbits, accn, acw, acv);
            if (g.active && ok) {
                if (!fixed) sptr[(size_t)pass * sstep] = sv;   // a fixed pass leaves it as it is
                xptr[(size_t)pass * xstep] = (uint8_t)xbits;
            }
            add_row_sums<kNarrow>(b.lanes, b.leader, ok, rr, accn, acw, acv, s_acc32, s_acc64);
        };

        // Three state buffers in rotation: two rows in flight while one is computed.
        uint4 sa = load_state(0), sb = load_state(1), sc;
        uint32_t xa = load_xold(0), xb1 = load_xold(1), xc = 0u;
        for (int pass = 0; pass < passes; pass += 3) {
            sc = load_state(pass + 2);
            xc = load_xold(pass + 2);
            process(sa, xa, pass);
            if (pass + 1 >= passes) break;
            sa = load_state(pass + 3);
            xa = load_xold(pass + 3);
            process(sb, xb1, pass + 1);
            if (pass + 2 >= passes) break;
            sb = load_state(pass + 4);
            xb1 = load_xold(pass + 4);
            process(sc, xc, pass + 2);
        }
        flush_segment<kNarrow>(p, t, ra, seg_rows, s_acc32, s_acc64);
    }
}

// ---------------------------------------------------------------------------------------
// Asynchronous-copy form (any tile shape). Each thread streams its own 16-byte vectors
// through a private ring of kRingStages shared-memory slots with cp.async: the copy for
// pass P + kRingStages - 1 is issued before pass P is computed and the thread waits only
// for its own copy groups, so kRingStages - 1 rows per thread are in flight without
// registers and without any block-wide synchronisation.
// ---------------------------------------------------------------------------------------
constexpr int kRingStages = 8;

__device__ __forceinline__ uint32_t smem_u32(const void *ptr)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(ptr));
}

// 16-byte global->shared copy; src_bytes = 0 writes zeros (nothing is read).
__device__ __forceinline__ void cp_async16(void *dst, const void *src, uint32_t src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
                 :: "r"(smem_u32(dst)), "l"(src), "r"(src_bytes) : "memory");
}

// 8-byte global->shared copy (byte state); src_bytes = 0 writes zeros.
__device__ __forceinline__ void cp_async8(void *dst, const void *src, uint32_t src_bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;"
                 :: "r"(smem_u32(dst)), "l"(src), "r"(src_bytes) : "memory");
}

// Byte state <-> the 16-bit lanes the kernels compute on: 8 bytes (4n of genes 0..7) to
// four words of two 16-bit halves, and back (every value is at most 8K <= 240).
__device__ __forceinline__ uint4 unpack8(uint2 w)
{
    return make_uint4(__byte_perm(w.x, 0u, 0x4140), __byte_perm(w.x, 0u, 0x4342),
                      __byte_perm(w.y, 0u, 0x4140), __byte_perm(w.y, 0u, 0x4342));
}

__device__ __forceinline__ uint2 pack8(uint4 v)
{
    return make_uint2(__byte_perm(v.x, v.y, 0x6420), __byte_perm(v.z, v.w, 0x6420));
}

__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory");
}

// One tile segment (rows ra .. ra + seg_rows - 1 of tile `tile`) of one generation. kS8:
// the state is stored as bytes (copied 8 bytes per pass, widened to 16-bit lanes).
// kSegDelta: rule R1 deltas formed once per segment into s_delta. The host selects it with
// the segment queue (long segments): measured on c3 358 vs 364 us per generation; with
// c2's short static segments it costs (9.99 vs 9.61 us), and the batched kernel, whose
// segments are many and short, forms the deltas every pass (4,618 vs 4,338 solves/s on c4).
// kUnroll2: the pass loop unrolled twice (the batched kernel: c4 4,692 vs 4,593 solves/s;
// no gain for the single-instance kernels, c2 9.90 vs 9.70 us per generation).
//
// kF: the instance keeps fixed-vector words (tiles of 256 vectors, one row per pass): every
// pass forms its F from its threshold words, each warp stores the 32 bits of its vectors as
// one word, and nfix counts the set ones.
// Both count in nskip the vectors that did not draw (the fixed-allele passes).
// kSample (an instance whose words are not kept yet): nfix counts 16 for every vector the
// fixed-allele test finds at the bounds (the test runs on about one pass in 16 while the
// population is spread), an estimate that decides when to start keeping them.
template <bool kNarrow, int kRule, bool kCip, class Keys, bool kS8 = false, bool kSegDelta = false,
          bool kUnroll2 = false, bool kF = false, bool kSample = false>
__device__ __forceinline__ void ring_segment(const GenParams &p, const Keys &keys, const BlockShare &b,
                                             int tile, int ra, int seg_rows, int32_t t,
                                             const uint8_t *x_prev, uint8_t *x_cur,
                                             const uint8_t *elite_row,
                                             const unsigned char *thr_bytes, uint4 *slots,
                                             uint32_t *s_acc32, unsigned long long *s_acc64,
                                             int &countdown, uint32_t *nfix = nullptr,
                                             uint32_t *nskip = nullptr)
{
    const int rpp = b.rows_per_pass;
    const int passes = (seg_rows + rpp - 1) / rpp;
    const int ra_key = ra + p.row0;             // chromosome index of row ra in the draws

    SegCtx g;
    seg_setup<kNarrow, kCip, kSegDelta>(p, g, tile, b.v_in, b.tile_vecs, elite_row);
    const size_t row0 = (size_t)ra + b.r_sub;
    using SV = typename std::conditional<kS8, uint2, uint4>::type;
    SV *sptr = reinterpret_cast<SV *>(p.state) + row0 * p.svec + g.vec;
    const size_t sstep = (size_t)rpp * p.svec;
    uint8_t *xptr = x_cur + row0 * p.xstride + g.vec;
    const uint8_t *xoptr = x_prev + row0 * p.xstride + g.vec;
    const size_t xstep = (size_t)rpp * p.xstride;

    // Incremental addressing (no multiplies in the pass loop): the copy cursor runs
    // kRingStages - 1 rows ahead of the compute cursor.
    const SV *ld_ptr = sptr;                    // next row to copy
    SV *st_ptr = sptr;                          // row being computed
    uint8_t *xst_ptr = xptr;
    const uint8_t *xo_ptr = xoptr;
    int rr = b.r_sub;
    uint32_t *fptr = nullptr;                   // kF: this warp's F word of row ra + rr
    if constexpr (kF) fptr = p.fword + (size_t)ra * (p.fstride >> 5) + (size_t)(g.vec >> 5);
    auto issue = [&](uint32_t stage, bool v) {
        if constexpr (kS8)
            cp_async8(slots + (size_t)stage * kThreads, v ? (const void *)ld_ptr : (const void *)p.state,
                      v ? 8u : 0u);
        else
            cp_async16(slots + (size_t)stage * kThreads, v ? (const void *)ld_ptr : (const void *)p.state,
                       v ? 16u : 0u);
        cp_async_commit();
        ld_ptr += sstep;
    };
    auto load_xold = [&](const uint8_t *ptr, int r) -> uint32_t {
        if (kRule != 1 || !kCip) return 0u;
        if (!(g.active && r < seg_rows)) return 0u;
        return (uint32_t)*ptr;
    };

#pragma unroll
    for (int k = 0; k < kRingStages - 1; ++k) issue((uint32_t)k, g.active && b.r_sub + k * rpp < seg_rows);
    const int lim = seg_rows - (kRingStages - 1) * rpp;
    uint32_t xa = load_xold(xo_ptr, rr), xb1 = load_xold(xo_ptr + xstep, rr + rpp);
#pragma unroll(kUnroll2 ? 2 : 1)
    for (int pass = 0; pass < passes; ++pass) {
        issue((uint32_t)(pass + kRingStages - 1) & (kRingStages - 1), g.active && rr < lim);
        const uint32_t xo = xa;
        xa = xb1;
        xb1 = load_xold(xo_ptr + 2 * xstep, rr + 2 * rpp);
        xo_ptr += xstep;
        cp_async_wait<kRingStages - 1>();
        uint4 sv;
        const uint32_t slot = (uint32_t)pass & (kRingStages - 1);
        if constexpr (kS8) sv = unpack8(*reinterpret_cast<const uint2 *>(slots + (size_t)slot * kThreads));
        else sv = slots[(size_t)slot * kThreads];

        const bool ok = rr < seg_rows;
        uint32_t xbits, accn, zor = 1u;
        int64_t acw, acv;
        bool fixed;
        sv = qubit_pass<kNarrow, kRule, kCip, Keys, kSegDelta>(p, keys, g, sv, xo, ra_key + rr, t, thr_bytes,
                                                               fixed, countdown, xbits, accn, acw, acv,
                                                               kF ? &zor : nullptr, kSample ? nfix : nullptr,
                                                               (kF || kSample) ? nskip : nullptr);
        if (g.active && ok) {
            if (!fixed) {               // a fixed pass leaves the state as it is
                if constexpr (kS8) *st_ptr = pack8(sv);
                else *st_ptr = sv;
            }
            *xst_ptr = (uint8_t)xbits;
        }
        if constexpr (kF) {
            const bool fx = g.active && ok && zor == 0u;
            const uint32_t fb = __ballot_sync(0xffffffffu, fx);
            if ((threadIdx.x & 31) == 0 && ok) *fptr = fb;
            *nfix += fx ? 1u : 0u;
            fptr += p.fstride >> 5;
        }
        add_row_sums<kNarrow>(b.lanes, b.leader, ok, rr, accn, acw, acv, s_acc32, s_acc64);
        st_ptr += sstep;
        xst_ptr += xstep;
        rr += rpp;
    }
    cp_async_wait<0>();
    flush_segment<kNarrow, (kF || kSample) ? 1 : 0>(p, t, ra, seg_rows, s_acc32, s_acc64);
}

// ---------------------------------------------------------------------------------------
// Sparse form of a tile segment (instances that keep F: packed sums, 16-bit state, tiles of
// 256 vectors; generations that rotate, i.e. not a run's first). Once most of the
// population has collapsed, most vectors are stable: every qubit at a bound on the side of
// the previous elite's allele, so CIP leaves it, the observation cannot differ from the
// side, the state needs no read or write, and the vector's alleles, hence its share of the
// row sums, are those of the generation before. Which vectors are unstable follows the
// columns (a gene where the elite left the consensus is unstable in nearly every row), so
// the warps split the segment by rows, not columns: warp w takes rows w, w + 8, ... and lane
// l the 8 consecutive vectors 8 l .. 8 l + 7 of the tile, so every warp meets the same
// columns and the same share of the work. Per row a warp:
//   1. reads F of its 256 vectors and their previous alleles (one byte and 8 bytes a lane,
//      loaded four rows ahead) and writes the stable vectors' alleles (their sides; one
//      8-byte store a lane); nothing else: the row's totals of the generation before
//      (fprev) already hold their share;
//   2. lists the row's unstable vectors in its slice of a shared-memory ring.
// It then streams the listed vectors' state through the per-thread cp.async ring, 32 per
// step, and runs the full pass on each (the
// vector's items and CIP steps are read from the slots of the thread that set up its
// column): CIP, QIP, the state, the alleles and F; its sums enter the row as the signed
// change against the previous alleles (shared atomics on the row's accumulators, which only
// this warp touches), and combine_row_delta adds them to the row's totals.
// Listing runs ahead of the copies, so the ring's 7 rows of look-ahead become 7 steps of
// 32 listed vectors. All sums are exact integers, so the results equal the dense form's.
// Segments hold at most 256 rows (a list entry holds the row, the vector, its previous
// alleles and its F bit, so that F is written only when it changes).
// ---------------------------------------------------------------------------------------
constexpr int kListCap = 512;               // entries of a warp's list (a power of two)
__shared__ uint32_t s_list[kThreads / 32][kListCap];
// The queue index and descriptor of a block's next segment in sparse generations (written by
// thread 0 during the current segment, read after its last barrier)
__shared__ int32_t s_next_qi;
__shared__ int4 s_next_sg;
__shared__ uint8_t s_e8[kThreads];          // rule R2: the previous elite's alleles of the tile's vectors

// Packed narrow sums (sum v << 16 | sum w) of 8 genes from their alleles (bit i = gene i)
// and the vector's item byte vectors.
__device__ __forceinline__ uint32_t narrow_sums_bits(uint32_t x8, uint4 ib)
{
    const uint32_t xa = allele_bytes(x8 & 15u), xb = allele_bytes((x8 >> 4) & 15u);
    const uint32_t sw = __dp4a(xa, ib.x, __dp4a(xb, ib.y, 0u));
    const uint32_t sv = __dp4a(xa, ib.z, __dp4a(xb, ib.w, 0u));
    return sw | (sv << 16);
}

// Bit k = (byte k of a == byte k of b), for the 8 bytes of two uint2: the zero bytes of the
// difference (0x80 in each, exactly: no carry crosses a byte), gathered by a multiply whose
// four terms move bit 7, 15, 23, 31 to bits 28-31 without carries.
__device__ __forceinline__ uint32_t equal_bytes8(uint2 a, uint2 b)
{
    const uint32_t d0 = a.x ^ b.x, d1 = a.y ^ b.y;
    const uint32_t z0 = ~(((d0 & 0x7f7f7f7fu) + 0x7f7f7f7fu) | d0 | 0x7f7f7f7fu);
    const uint32_t z1 = ~(((d1 & 0x7f7f7f7fu) + 0x7f7f7f7fu) | d1 | 0x7f7f7f7fu);
    return (((z0 >> 7) * 0x10204080u) >> 28) | ((((z1 >> 7) * 0x10204080u) >> 28) << 4);
}

// Rows of F and previous alleles a warp of the sparse form has in flight.
constexpr int kSparseAhead = 4;

template <int kRule>
__device__ __forceinline__ void sparse_segment(const GenParams &p, int tile, int ra, int seg_rows, int32_t t,
                                               const uint8_t *x_prev, uint8_t *x_cur, const uint8_t *elite_row,
                                               const unsigned char *thr_bytes, uint4 *slots,
                                               uint32_t *s_acc32, uint32_t *list, uint32_t &nfix,
                                               uint32_t &nskip, int32_t next)
{
    constexpr uint32_t kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const uint32_t off_top = (uint32_t)(8 * p.K);
    const uint32_t k8 = off_top * 0x00010001u;
    const uint32_t ra_key = (uint32_t)(ra + p.row0);
    const size_t svec = (size_t)p.svec, xstride = (size_t)p.xstride, fstride = (size_t)p.fstride;
    const uint32_t vt = (uint32_t)tile * kThreads;              // the tile's first vector
    const uint32_t vb = vt + 8u * (uint32_t)lane;               // this lane's first vector
    const int nact = max(0, min(8, (int)((int64_t)svec - (int64_t)vb)));   // of its 8, active
    const int nrows = seg_rows > warp ? (seg_rows - warp + 7) >> 3 : 0;     // this warp's rows

    // F and the previous alleles of this warp's next rows in flight (one row's work is too
    // short to cover a load's latency); the first loads go out before the segment's others.
    // A lane's 8 vectors have 8 bits of F: byte l of the tile's 8 words of the row.
    const uint8_t *fsrc = reinterpret_cast<const uint8_t *>(p.fword + (size_t)(ra + warp) * (fstride >> 5) +
                                                            (vt >> 5)) + lane;
    const uint2 *xsrc = reinterpret_cast<const uint2 *>(x_prev + (size_t)(ra + warp) * xstride + vb);
    // 8 rows in bytes / uint2 units; both below 2^32, so each address is one 32 x 32 -> 64
    // multiply-add
    const uint32_t fstep = (uint32_t)fstride, xstep = (uint32_t)xstride;
    const int mlim = nact > 0 ? nrows : 0;      // rows this lane loads
    auto fload = [&](int m) -> uint32_t {
        return m < mlim ? (uint32_t)__ldcg(fsrc + (size_t)(uint32_t)m * (size_t)fstep) : 0u;
    };
    auto xload = [&](int m) -> uint2 {
        return m < mlim ? __ldcg(xsrc + (size_t)(uint32_t)m * (size_t)xstep) : make_uint2(0u, 0u);
    };
    uint32_t fb[kSparseAhead];                  // slot i: row m + ((i - m) mod kSparseAhead)
    uint2 xb[kSparseAhead];
#pragma unroll
    for (int i = 0; i < kSparseAhead; ++i) {
        fb[i] = fload(i);
        xb[i] = xload(i);
    }

    SegCtx g;
    seg_setup<true, true, kRule == 0>(p, g, tile, threadIdx.x, kThreads, elite_row);
    if (kRule == 1) s_e8[threadIdx.x] = (uint8_t)g.e8;
    // this lane's 8 elite alleles: a vector is stable when it is fixed and its previous
    // alleles (its sides) equal them
    uint2 e8s = make_uint2(0u, 0u);
    if (nact > 0) e8s = __ldcg(reinterpret_cast<const uint2 *>(elite_row + vb));
    const uint32_t vmask = (1u << nact) - 1u;
    __syncthreads();                            // every thread reads the slots of the block's columns
    uint4 *const sbase = p.state + (size_t)ra * svec + vt;      // row ra, the tile's vector 0
    uint8_t *const xbase = x_cur + (size_t)ra * xstride + vt;
    uint8_t *const xlane = xbase + 8u * (uint32_t)lane;         // this lane's alleles, row 0

    int m = 0;                                  // this warp's rows listed so far
    uint32_t head = 0;                          // entries listed so far (warp-uniform)

    // Steps 1 and 2 for this warp's next row (row = warp + 8 m of the segment). A list entry
    // is row << 17 | (F was set) << 16 | previous alleles << 8 | vector of the tile.
    auto produce = [&](uint32_t &fslot, uint2 &xslot) {
        const uint32_t fbits = fslot;
        const uint2 xo = xslot;
        fslot = fload(m + kSparseAhead);        // the slot's next row
        xslot = xload(m + kSparseAhead);
        const int row = warp + 8 * m;
        ++m;
        const uint32_t sm = fbits & equal_bytes8(xo, e8s) & vmask;
        const uint32_t um = vmask & ~sm;
        const uint32_t ns = (uint32_t)__popc(sm);
        nfix += ns;
        nskip += ns;
        // The stable vectors' alleles; with all 8 vectors active, the unstable ones' bytes go
        // too and are overwritten by their own pass after the __syncwarp that ends the listing
        uint8_t *xp = xlane + (size_t)(uint32_t)row * (size_t)xstep;
        if (nact == 8 && sm != 0u) {
            *reinterpret_cast<uint2 *>(xp) = e8s;
        } else if (sm != 0u) {
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if ((sm >> k) & 1u) xp[k] = (uint8_t)((k < 4 ? e8s.x : e8s.y) >> (8 * (k & 3)));
        }
        // the row's unstable vectors, in lane order (an exclusive prefix sum of the counts)
        const uint32_t cnt = (uint32_t)__popc(um);
        if (__any_sync(kFull, cnt != 0u)) {
            uint32_t pre = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(kFull, pre, o);
                if (lane >= o) pre += y;
            }
            const uint32_t total = __shfl_sync(kFull, pre, 31);
            uint32_t pos = head + pre - cnt;
            uint32_t bits = um;
            while (bits != 0u) {
                const int k = __ffs((int)bits) - 1;
                bits &= bits - 1u;
                const uint32_t xk = ((k < 4 ? xo.x : xo.y) >> (8 * (k & 3))) & 0xffu;
                list[pos & (kListCap - 1)] = ((uint32_t)row << 17) | (((fbits >> k) & 1u) << 16) | (xk << 8) |
                                             (8u * (uint32_t)lane + (uint32_t)k);
                ++pos;
            }
            head += total;
        }
    };

    // Lists rows while m < nrows and head < lim. Row m sits in slot m % 4: a slot is read
    // once, when its row is listed, and refilled at once, so each load stays in flight for
    // four rows (moving the window through the registers would wait for every load at the
    // next row).
    static_assert(kSparseAhead == 4, "slots are selected by m % 4");
    auto list_rows = [&](uint32_t lim) {
#pragma unroll 1
        for (;;) {
            switch (m & 3) {
            case 0: if (!(m < nrows && head < lim)) return; produce(fb[0], xb[0]); [[fallthrough]];
            case 1: if (!(m < nrows && head < lim)) return; produce(fb[1], xb[1]); [[fallthrough]];
            case 2: if (!(m < nrows && head < lim)) return; produce(fb[2], xb[2]); [[fallthrough]];
            default: if (!(m < nrows && head < lim)) return; produce(fb[3], xb[3]);
            }
        }
    };

    // Copies of step j (entries 32 j .. 32 j + 31) into ring slot j % 8; the step must be
    // listed in full (or the listing finished).
    auto issue = [&](uint32_t j) {
        const uint32_t i = j * 32u + (uint32_t)lane;
        const bool has = i < head;
        const void *src = p.state;
        if (has) {
            const uint32_t e = list[i & (kListCap - 1)];
            src = sbase + (size_t)(e >> 17) * svec + (e & 255u);
        }
        cp_async16(slots + (size_t)(j & (kRingStages - 1)) * kThreads, src, has ? 16u : 0u);
        cp_async_commit();
    };

    // Step 3 for step j; each vector's change goes to its row with two shared atomics.
    auto compute = [&](uint32_t j) {
        const uint32_t i = j * 32u + (uint32_t)lane;
        if (i >= head) return;
        const uint32_t e = list[i & (kListCap - 1)];
        const uint32_t row = e >> 17;
        const uint32_t col = e & 255u;
        const uint32_t xo = (e >> 8) & 0xffu;
        const uint32_t vec = vt + col;
        uint4 s = slots[(size_t)(j & (kRingStages - 1)) * kThreads];
        if (kRule == 0) {                       // R1: every qubit toward the elite's allele
            const uint4 d = s_delta[col];
            s.x = rotate_pair_signed(s.x, d.x, k8);
            s.y = rotate_pair_signed(s.y, d.y, k8);
            s.z = rotate_pair_signed(s.z, d.z, k8);
            s.w = rotate_pair_signed(s.w, d.w, k8);
        } else {                                // R2: the qubits whose allele differed
            const uint32_t e8c = s_e8[col];
            s = rotate_vec(s, e8c, e8c ^ xo, k8);
        }
        const Draw4 r0 = philox4x32_10_rk(2u * vec, ra_key + row, (uint32_t)t, 0u, p.rk0, p.rk1);
        const Draw4 r1 = philox4x32_10_rk(2u * vec + 1u, ra_key + row, (uint32_t)t, 0u, p.rk0, p.rk1);
        const uint32_t u[8] = {r0.a, r0.b, r0.c, r0.d, r1.a, r1.b, r1.c, r1.d};
        const uint32_t sp[4] = {s.x, s.y, s.z, s.w};
        uint32_t xbits = 0u, z = 0u;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint32_t off = (k & 1) ? (sp[k >> 1] >> 16) : (sp[k >> 1] & 0xffffu);
            const uint32_t thr = *reinterpret_cast<const uint32_t *>(thr_bytes + off);
            z |= thr;
            if ((u[k] < thr) || (off == off_top)) xbits |= 1u << k;
        }
        if (xbits != xo) {
            const uint4 ib = s_item_bytes[col];
            const uint32_t a = narrow_sums_bits(xbits, ib), b = narrow_sums_bits(xo, ib);
            atomicAdd(s_acc32 + 2 * row, (a & 0xffffu) - (b & 0xffffu));
            atomicAdd(s_acc32 + 2 * row + 1, (a >> 16) - (b >> 16));
        }
        sbase[(size_t)row * svec + col] = s;
        xbase[(size_t)row * xstride + col] = (uint8_t)xbits;
        const uint32_t fx = z == 0u ? 1u : 0u;
        if (fx != ((e >> 16) & 1u)) {            // F changed: set or clear this vector's bit
            uint32_t *w = p.fword + ((size_t)ra + row) * (fstride >> 5) + (vec >> 5);
            if (fx) atomicOr(w, 1u << (vec & 31u));
            else atomicAnd(w, ~(1u << (vec & 31u)));
        }
        nfix += fx;
    };

    // Listing runs ahead of the copies in bursts: the steps up to jc + 7 are listed before
    // the copies of jc + 7 are issued, and a burst stops once they are, so the live entries
    // (from step jc on) stay below 32 (jc + 8) + 256 <= 32 jc + 512, the list's size. The
    // loop between bursts issues and computes without listing.
    list_rows(8u * 32u);
    __syncwarp();
    // thread 0: the next segment's descriptor (its index, taken at the segment's start, has
    // arrived by now), published before the flush's last barrier
    int4 sg_next = make_int4(0, 0, 0, 0);
    if (threadIdx.x == 0 && next < p.nsegs) sg_next = __ldg(p.segq + next);
    const bool any = m < nrows || head != 0u;   // else every row was stable: no copies
#pragma unroll 1
    for (uint32_t j = 0; any && j < kRingStages - 1; ++j) issue(j);
    uint32_t jc = 0;
#pragma unroll 1
    while (any) {
        list_rows((jc + 8u) * 32u);
        __syncwarp();
        const bool done = m >= nrows;
        const uint32_t avail = done ? (head + 31u) / 32u : head / 32u;
        if (jc >= avail) break;
        const uint32_t jend = done ? avail : avail - (kRingStages - 1);
#pragma unroll 1
        for (; jc < jend; ++jc) {
            issue(jc + kRingStages - 1);
            cp_async_wait<kRingStages - 1>();
            compute(jc);
        }
    }
    cp_async_wait<0>();
    if (threadIdx.x == 0) {      // every thread read the current ones before the setup barrier
        s_next_qi = next;
        s_next_sg = sg_next;
    }
    flush_segment<true, 2>(p, t, ra, seg_rows, s_acc32, nullptr, tile);
}

template <bool kNarrow>
__device__ __forceinline__ void clear_row_sums(int seg_rows_max, uint32_t *s_acc32,
                                               unsigned long long *s_acc64)
{
    for (int i = threadIdx.x; i < 2 * seg_rows_max; i += kThreads) {
        if (kNarrow) s_acc32[i] = 0u;
        else s_acc64[i] = 0ull;
    }
    __syncthreads();
}

template <bool kNarrow, int kRule, bool kCip, bool kS8 = false, bool kSegDelta = false>
__device__ __forceinline__ void generation_body_ring(const GenParams &p, const BlockShare &b,
                                                     int32_t t, int32_t e_prev, uint4 *ring,
                                                     const uint32_t *s_thr, uint32_t *s_acc32,
                                                     unsigned long long *s_acc64)
{
    const unsigned char *thr_bytes = reinterpret_cast<const unsigned char *>(s_thr);
    const uint8_t *x_prev = p.xbits + (size_t)((t + 1) & 1) * p.xplane;
    uint8_t *x_cur = p.xbits + (size_t)(t & 1) * p.xplane;
    const uint8_t *elite_row = x_prev + (size_t)e_prev * p.xstride;
    uint4 *slots = ring + threadIdx.x;           // slot s of this thread: slots[s * kThreads]
    int countdown = 0;
    clear_row_sums<kNarrow>(p.seg_rows_max, s_acc32, s_acc64);
    for (int64_t u0 = b.u_begin; u0 < b.u_end;) {
        const int tile = (int)(u0 / p.np);
        const int ra = (int)(u0 - (int64_t)tile * p.np);
        const int seg_rows = (int)min(min((int64_t)(p.np - ra), b.u_end - u0), (int64_t)p.seg_rows_max);
        u0 += seg_rows;
        ring_segment<kNarrow, kRule, kCip, ParamKeys, kS8, kSegDelta>(p, ParamKeys{p}, b, tile, ra, seg_rows, t,
                                                                      x_prev, x_cur, elite_row, thr_bytes, slots,
                                                                      s_acc32, s_acc64, countdown);
    }
}

// One generation over segments taken from the instance's queue (deferred forms). The blocks
// that share an SM do not get equal issue slots (the schedulers favour older warps), so
// with equal static shares the blocks launched first finish early and leave their SM part
// empty while the others finish; taken from a queue in order of decreasing size, the
// segments keep every block busy until the work runs out. Any split gives the same
// results: each tile-row's sums are exact integers added once per segment.
//
// kF (instances that can keep F). While fcnt[3] is 0 the words are not kept: they are all 0
// (cleared with the state and never written since), the dense form runs as without them and
// estimates the fixed vectors from the fixed-allele test's samples. Once that estimate
// reaches f_on_min the words are kept from then on (fcnt[3] = 1, set by block 0 of the
// first such generation): the dense form writes every vector's F, and a generation takes the
// sparse form (sparse_segment) when at least sparse_min vectors were fixed after the one
// before. Each warp adds its count (exact, or the estimate) to fcnt[t % 3].
template <bool kNarrow, int kRule, bool kCip, bool kS8 = false, bool kSegDelta = false, bool kF = false>
__device__ __forceinline__ void generation_body_queue(const GenParams &p, const BlockShare &b,
                                                      int32_t t, int32_t e_prev, uint4 *ring,
                                                      const uint32_t *s_thr, uint32_t *s_acc32,
                                                      unsigned long long *s_acc64)
{
    __shared__ int32_t s_qi;
    const unsigned char *thr_bytes = reinterpret_cast<const unsigned char *>(s_thr);
    const uint8_t *x_prev = p.xbits + (size_t)((t + 1) & 1) * p.xplane;
    uint8_t *x_cur = p.xbits + (size_t)(t & 1) * p.xplane;
    const uint8_t *elite_row = x_prev + (size_t)e_prev * p.xstride;
    uint4 *slots = ring + threadIdx.x;
    unsigned int *ctr = p.qctr + (t % 3);
    int countdown = 0;
    uint32_t nfix = 0u, nskip = 0u;
    bool keep = false, sparse = false;
    __shared__ unsigned long long s_cnt[2];
    if constexpr (kF) {
        const unsigned long long prev = __ldcg(p.fcnt + (t + 2) % 3);
        keep = __ldcg(p.fcnt + 3) != 0ull || prev >= p.f_on_min;
        sparse = kCip && keep && prev >= p.sparse_min;
        if (keep && blockIdx.x == 0 && threadIdx.x == 0) p.fcnt[3] = 1ull;
        if (threadIdx.x == 0) s_cnt[0] = s_cnt[1] = 0ull;   // read after the loop's barriers
    }
    clear_row_sums<kNarrow>(p.seg_rows_max, s_acc32, s_acc64);
    // Sparse generations: thread 0 takes the next segment's index while the block works on
    // the current one (the atomic's round trip is off the block's path; a sparse
    // segment's work is short), loads its descriptor once the index has arrived, and
    // publishes both before the segment's last barrier (the flush's), which every thread
    // passes before reading them. Dense ones take the index when they need it (holding a
    // second segment would coarsen the end of the guided schedule).
    if (threadIdx.x == 0) {
        s_qi = (int32_t)atomicAdd(ctr, 1u);
        if (kF && sparse && s_qi < p.nsegs) s_next_sg = __ldg(p.segq + s_qi);
    }
    __syncthreads();
    int32_t qi = s_qi;
    for (;;) {
        if (qi >= p.nsegs) break;
        int32_t next = 0;
        if (sparse && threadIdx.x == 0) next = (int32_t)atomicAdd(ctr, 1u);
        const int4 sg = (kF && sparse) ? s_next_sg : __ldg(p.segq + qi);
        if constexpr (kF) {
            if (sparse)
                sparse_segment<kRule>(p, sg.x, sg.y, sg.z, t, x_prev, x_cur, elite_row, thr_bytes, slots,
                                      s_acc32, s_list[threadIdx.x >> 5], nfix, nskip, next);
            else if (keep)
                ring_segment<kNarrow, kRule, kCip, ParamKeys, kS8, kSegDelta, false, true>(
                    p, ParamKeys{p}, b, sg.x, sg.y, sg.z, t, x_prev, x_cur, elite_row, thr_bytes, slots, s_acc32,
                    s_acc64, countdown, &nfix, &nskip);
            else
                ring_segment<kNarrow, kRule, kCip, ParamKeys, kS8, kSegDelta, false, false, true>(
                    p, ParamKeys{p}, b, sg.x, sg.y, sg.z, t, x_prev, x_cur, elite_row, thr_bytes, slots, s_acc32,
                    s_acc64, countdown, &nfix, &nskip);
        } else {
            ring_segment<kNarrow, kRule, kCip, ParamKeys, kS8, kSegDelta>(p, ParamKeys{p}, b, sg.x, sg.y, sg.z, t,
                                                                          x_prev, x_cur, elite_row, thr_bytes,
                                                                          slots, s_acc32, s_acc64, countdown);
        }
        if (kF && sparse) {
            qi = s_next_qi;             // published before the flush's last barrier
        } else {
            // every thread has read the index before the segment's first barrier
            if (threadIdx.x == 0) s_qi = (int32_t)atomicAdd(ctr, 1u);
            __syncthreads();
            qi = s_qi;
        }
    }
    if constexpr (kF) {
        // one atomic per block for each count
        const uint32_t n = __reduce_add_sync(0xffffffffu, nfix), d = __reduce_add_sync(0xffffffffu, nskip);
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&s_cnt[0], (unsigned long long)n);
            atomicAdd(&s_cnt[1], (unsigned long long)d);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (s_cnt[0] != 0ull) atomicAdd(p.fcnt + t % 3, s_cnt[0]);
            if (s_cnt[1] != 0ull) atomicAdd(p.fcnt + 4 + t % 3, s_cnt[1]);
        }
    }
}

// CIP with elite e of generation t over this block's share (the final rotation of a run).
template <int kRule, bool kS8 = false>
__device__ __forceinline__ void final_cip_body(const GenParams &p, const BlockShare &b,
                                               int32_t t, int32_t e)
{
    const uint8_t *xl = p.xbits + (size_t)(t & 1) * p.xplane;
    const uint8_t *elite_row = xl + (size_t)e * p.xstride;
    const uint32_t k8 = (uint32_t)(8 * p.K) * 0x00010001u;
    for (int64_t u0 = b.u_begin; u0 < b.u_end;) {
        const int tile = (int)(u0 / p.np);
        const int ra = (int)(u0 - (int64_t)tile * p.np);
        const int seg_rows = (int)min(min((int64_t)(p.np - ra), b.u_end - u0), (int64_t)p.seg_rows_max);
        u0 += seg_rows;
        const int vec = tile * b.tile_vecs + b.v_in;
        if (vec >= p.svec) continue;
        const uint32_t e8 = __ldcg(elite_row + vec);
        // four rows per step, loads first
        for (int rr = b.r_sub; rr < seg_rows; rr += 4 * b.rows_per_pass) {
            uint4 v[4];
            uint32_t m8[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int r2 = rr + k * b.rows_per_pass;
                if (r2 < seg_rows) {
                    const size_t c = (size_t)ra + r2;
                    if constexpr (kS8) v[k] = unpack8(reinterpret_cast<const uint2 *>(p.state)[c * p.svec + vec]);
                    else v[k] = p.state[c * p.svec + vec];
                    m8[k] = kRule == 1 ? (e8 ^ (uint32_t)xl[c * p.xstride + vec]) : 0xffu;
                }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int r2 = rr + k * b.rows_per_pass;
                if (r2 < seg_rows) {
                    const size_t i = ((size_t)ra + r2) * p.svec + vec;
                    const uint4 r = rotate_vec(v[k], e8, m8[k], k8);
                    if constexpr (kS8) reinterpret_cast<uint2 *>(p.state)[i] = pack8(r);
                    else p.state[i] = r;
                }
            }
        }
    }
}

// Bounded grid barrier after generation t: the last block to arrive closes the generation
// and releases the others. Returns false when the wait ran out or an error was raised
// (the block then stops; the host reports QIEO_ERR_TIMEOUT).
__device__ __forceinline__ bool generation_barrier(const GenParams &p, int32_t t)
{
    __shared__ int s_flag;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int prev = atomicAdd(p.ticket, 1u);
        s_flag = (prev == gridDim.x - 1u) ? 1 : 0;
    }
    __syncthreads();
    if (s_flag) {
        __threadfence();
        close_generation(p, t);
        if (threadIdx.x == 0) {
            *p.ticket = 0u;
            *p.gen = t + 1;
            __threadfence();
            st_release(p.bar_gen, t + 1);
        }
    } else if (threadIdx.x == 0) {
        const uint64_t deadline = global_ns() + p.wait_ns;
        int ok = 0;
        for (uint32_t it = 0; it < (1u << 30); ++it) {
            if (ld_acquire(p.bar_gen) >= t + 1) {
                ok = 1;
                break;
            }
            if (ld_acquire(p.error) != 0 || global_ns() > deadline) break;
            __nanosleep(64);
        }
        if (!ok) atomicOr(p.error, kErrBarrierTimeout);
        s_flag = ok ? 2 : 0;
    }
    __syncthreads();
    return s_flag != 0;
}

// Plain grid barrier of a cooperative deferred-close run: each block's arrival is one
// release add to p.ticket (after a block barrier, so the add publishes every thread's
// writes); a block waits, bounded, until `target` arrivals are visible.
__device__ __forceinline__ void grid_arrive(const GenParams &p)
{
    __syncthreads();
    if (threadIdx.x == 0)
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" :: "l"(p.ticket) : "memory");
}

// kSpin: poll without sleeping (the resident form, whose generations are short).
template <bool kSpin = false>
__device__ __forceinline__ bool grid_wait(const GenParams &p, unsigned int target)
{
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        const uint64_t deadline = global_ns() + p.wait_ns;
        int ok = 0;
        for (uint32_t it = 0; it < (1u << 30); ++it) {
            if (ld_acquire(reinterpret_cast<const int32_t *>(p.ticket)) >= (int32_t)target) {
                ok = 1;
                break;
            }
            if (ld_acquire(p.error) != 0 || global_ns() > deadline) break;
            if (!kSpin) __nanosleep(32);
        }
        if (!ok) atomicOr(p.error, kErrBarrierTimeout);
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Dynamic shared memory: [per-thread copy ring (kRingStages x kThreads x 16 B)] when the
// asynchronous-copy form is used, then the per-row sums of a segment.
constexpr size_t kRingBytes = (size_t)kRingStages * kThreads * 16;

struct SmemParts {
    uint4 *ring;
    uint32_t *acc32;
    unsigned long long *acc64;
};

template <bool kRing>
__device__ __forceinline__ SmemParts carve_smem(unsigned char *raw)
{
    SmemParts m;
    m.ring = reinterpret_cast<uint4 *>(raw);
    unsigned char *acc = raw + (kRing ? kRingBytes : 0);
    m.acc32 = reinterpret_cast<uint32_t *>(acc);
    m.acc64 = reinterpret_cast<unsigned long long *>(acc);
    return m;
}

// queued: take the segments from the instance's queue (deferred forms with a queue).
template <bool kNarrow, int kRule, bool kCip, bool kRing, bool kS8 = false, bool kSegDelta = false,
          bool kF = false>
__device__ __forceinline__ void one_generation(const GenParams &p, const BlockShare &b, int32_t t,
                                               int32_t e_prev, SmemParts &m, const uint32_t *s_thr,
                                               bool queued = false)
{
    if constexpr (kRing) {
        if (queued && p.nsegs > 0)
            generation_body_queue<kNarrow, kRule, kCip, kS8, kSegDelta, kF>(p, b, t, e_prev, m.ring, s_thr,
                                                                            m.acc32, m.acc64);
        else
            generation_body_ring<kNarrow, kRule, kCip, kS8, kSegDelta>(p, b, t, e_prev, m.ring, s_thr,
                                                                       m.acc32, m.acc64);
    } else {
        generation_body<kNarrow, kRule, kCip>(p, b, t, e_prev, s_thr, m.acc32, m.acc64);
    }
}

// Records of generation t with elite e of fitness f: the history, the elite index, the
// best-so-far record (its row copied on a strict improvement) and, with the convergence
// test, the run length of equal elite fitness ending at t. Called by all threads of one
// block; returns that run length (0 when the test is off).
__device__ int32_t record_generation(const GenParams &p, int32_t t, int32_t e, int64_t f)
{
    __shared__ int32_t s_improved, s_run;
    if (threadIdx.x == 0) {
        const int64_t best_f = __ldcg(p.best), best_g = __ldcg(p.best + 1);
        p.hist_e[t] = e;
        p.hist_f[t] = f;
        *p.elite_idx = e;
        const int improved = (best_g < 0 || f > best_f) ? 1 : 0;
        if (improved) {
            p.best[0] = f;
            p.best[1] = t;
            p.best[2] = e;
        }
        int32_t run = 0;
        if (p.converge) {
            const int32_t prev = t > 0 ? p.conv[(t - 1) & 1] : 0;
            run = (prev > 0 && f == p.hist_f[t - 1]) ? prev + 1 : 1;
            p.conv[t & 1] = run;
        }
        s_improved = improved;
        s_run = run;
    }
    __syncthreads();
    if (s_improved) {
        const uint4 *src = reinterpret_cast<const uint4 *>(
            p.xbits + (size_t)(t & 1) * p.xplane + (size_t)e * p.xstride);
        uint4 *dst = reinterpret_cast<uint4 *>(p.best_row);
        for (int i = threadIdx.x; i < p.xstride / 16; i += kThreads) dst[i] = __ldcg(src + i);
    }
    const int32_t run = s_run;
    __syncthreads();
    return run;
}

// Elite of generation t from its key slot (every row of t has been folded into it).
__device__ __forceinline__ void elite_from_key(const GenParams &p, int32_t t, int32_t &e, int64_t &f)
{
    const unsigned long long k = __ldcg(key_slot(p, t));
    e = (int32_t)(0xffffffu - (uint32_t)(k & 0xffffffull));
    f = (int64_t)(k >> 24) - kKeyBias;
    if (e < 0 || e >= p.np) {   // every row finishes in every generation; see close_generation
        if (blockIdx.x == 0) atomicOr(p.error, kErrEliteRange);
        e = 0;
    }
}

// Stop state of a deferred-close launch at generation t: 1 when the instance stopped
// before this launch's work (at a run's first generation: stopped at all; later: stopped
// at a generation <= t - 2, whose CIP an earlier launch applied).
__device__ __forceinline__ int deferred_skip(const GenParams &p, int32_t t)
{
    if (!p.converge) return 0;
    const int32_t state = ld_acquire(p.conv + 2);
    if (state != kStopped) return 0;
    return (p.g == 0 || *(volatile const int32_t *)(p.conv + 3) <= t - 2) ? 1 : 0;
}

// ---------------------------------------------------------------------------------------
// run_kernel: generations t0 .. t0+G-1 and the final CIP in one cooperative launch. The
// first generation applies no CIP (a run starts from a rotated state or from t = 0).
// ---------------------------------------------------------------------------------------
template <bool kNarrow, int kRule, bool kRing>
__global__ void __launch_bounds__(kThreads, kNarrow ? (kRing ? 4 : 3) : 2) run_kernel(const GenParams p, int32_t G)
{
    __shared__ uint32_t s_thr[kMaxThr];
    extern __shared__ __align__(128) unsigned char smem_raw[];
    SmemParts m = carve_smem<kRing>(smem_raw);
    load_thresholds(p, s_thr);
    grid_dependency_wait();
    __syncthreads();
    const BlockShare b = block_share(p);
    const int32_t t0 = *p.gen;
    int32_t e = 0;
    if (p.deferred) {
        // Deferred close: a plain grid barrier between generations (arrivals counted in
        // p.ticket over the whole run, cleared by the end-of-run launch); after it every
        // block reads the elite of the generation before from its key slot, and block 0
        // writes that generation's records.
        __shared__ int s_e;
        __shared__ long long s_f;
        for (int32_t g = 0; g <= G; ++g) {
            const int32_t t = t0 + g;
            int64_t f = 0;
            if (g > 0) {
                if (!grid_wait(p, (unsigned int)g * gridDim.x)) return;
                if (threadIdx.x == 0) {
                    int32_t ee;
                    int64_t ff;
                    elite_from_key(p, t - 1, ee, ff);
                    s_e = ee;
                    s_f = ff;
                }
                __syncthreads();
                e = s_e;
                f = s_f;
                if (blockIdx.x == 0) record_generation(p, t - 1, e, f);
            }
            if (g == G) break;
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                *key_slot(p, t + 1) = 0ull;
                p.qctr[(t + 1) % 3] = 0u;
            }
            if (g == 0) one_generation<kNarrow, kRule, false, kRing>(p, b, t, 0, m, s_thr, true);
            else one_generation<kNarrow, kRule, true, kRing>(p, b, t, e, m, s_thr, true);
            grid_arrive(p);
        }
        final_cip_body<kRule>(p, b, t0 + G - 1, e);
        return;
    }
    for (int32_t g = 0; g < G; ++g) {
        const int32_t t = t0 + g;
        if (g == 0) one_generation<kNarrow, kRule, false, kRing>(p, b, t, 0, m, s_thr);
        else one_generation<kNarrow, kRule, true, kRing>(p, b, t, e, m, s_thr);
        if (!generation_barrier(p, t)) return;
        e = __ldcg(p.elite_idx);
    }
    final_cip_body<kRule>(p, b, t0 + G - 1, e);
}

// ---------------------------------------------------------------------------------------
// Sixteen genes per thread and pass: two adjacent 8-gene vectors of a row (32 contiguous
// bytes of state). The per-gene arithmetic is that of qubit_pass; the per-pass work around
// it -- the copy ring's issue and wait, the countdown, the row-sum reduction, the pointer
// steps -- is shared by sixteen genes instead of eight. Rule R1 with the segment's signed
// steps, packed item sums with items <= 127 (32 lanes x 16 genes x 127 < 2^16), 16-bit
// state; a tile-row is 256 threads x 2 vectors, one row per pass.
// ---------------------------------------------------------------------------------------
constexpr int kRing2Stages = 8;
__shared__ uint4 s_item_bytes2[kThreads];   // the second vector's byte vectors
__shared__ uint4 s_delta2[kThreads];        // the second vector's signed steps

struct SegCtx2 {
    uint32_t wv[16];              // packed items (v << 16 | w) of the 16 genes
    uint32_t e0, e1;              // elite alleles of the two vectors
    uint32_t ctr0;                // Philox counter word 0 of the first 4 genes
    int vec;                      // the first vector (even)
    bool act0, act1;              // vec < svec, vec + 1 < svec
};

template <bool kCip>
__device__ __forceinline__ void seg_setup2(const GenParams &p, SegCtx2 &g, int tile, const uint8_t *elite_row)
{
    g.vec = tile * (2 * kThreads) + 2 * (int)threadIdx.x;
    g.act0 = g.vec < p.svec;
    g.act1 = g.vec + 1 < p.svec;
    const uint4 z = make_uint4(0, 0, 0, 0);
    uint4 a = z, c = z, d = z, a1 = z, c1 = z, d1 = z;
    if (g.act0) {
        a = __ldg(p.items_narrow + 2 * (size_t)g.vec);
        c = __ldg(p.items_narrow + 2 * (size_t)g.vec + 1);
        d = __ldg(p.items_narrow + 2 * (size_t)p.svec + g.vec);
    }
    if (g.act1) {
        a1 = __ldg(p.items_narrow + 2 * (size_t)g.vec + 2);
        c1 = __ldg(p.items_narrow + 2 * (size_t)g.vec + 3);
        d1 = __ldg(p.items_narrow + 2 * (size_t)p.svec + g.vec + 1);
    }
    g.wv[0] = a.x; g.wv[1] = a.y; g.wv[2] = a.z; g.wv[3] = a.w;
    g.wv[4] = c.x; g.wv[5] = c.y; g.wv[6] = c.z; g.wv[7] = c.w;
    g.wv[8] = a1.x; g.wv[9] = a1.y; g.wv[10] = a1.z; g.wv[11] = a1.w;
    g.wv[12] = c1.x; g.wv[13] = c1.y; g.wv[14] = c1.z; g.wv[15] = c1.w;
    s_item_bytes[threadIdx.x] = d;      // read back by this thread only
    s_item_bytes2[threadIdx.x] = d1;
    g.e0 = (kCip && g.act0) ? (uint32_t)__ldcg(elite_row + g.vec) : 0u;
    g.e1 = (kCip && g.act1) ? (uint32_t)__ldcg(elite_row + g.vec + 1) : 0u;
    if (kCip) {
        s_delta[threadIdx.x] = make_uint4(signed_step(delta_pair(g.e0 & 3u, 3u)),
                                          signed_step(delta_pair((g.e0 >> 2) & 3u, 3u)),
                                          signed_step(delta_pair((g.e0 >> 4) & 3u, 3u)),
                                          signed_step(delta_pair((g.e0 >> 6) & 3u, 3u)));
        s_delta2[threadIdx.x] = make_uint4(signed_step(delta_pair(g.e1 & 3u, 3u)),
                                           signed_step(delta_pair((g.e1 >> 2) & 3u, 3u)),
                                           signed_step(delta_pair((g.e1 >> 4) & 3u, 3u)),
                                           signed_step(delta_pair((g.e1 >> 6) & 3u, 3u)));
    }
    g.ctr0 = 2u * (uint32_t)g.vec;
}

// The saturation test of one vector: sat, and its alleles as the byte pair (xa, xb) and
// the byte xs (see qubit_pass).
__device__ __forceinline__ bool saturated_vec(uint4 s, uint32_t off_top, int bp, uint32_t &xa, uint32_t &xb,
                                              uint32_t &xs)
{
    const uint32_t b0 = (s.x >> bp) & 0x00010001u, b1 = (s.y >> bp) & 0x00010001u;
    const uint32_t b2 = (s.z >> bp) & 0x00010001u, b3 = (s.w >> bp) & 0x00010001u;
    xa = b0 | (b1 << 8);
    xb = b2 | (b3 << 8);
    xs = (allele_nibble_hi(xa) >> 24) | ((allele_nibble_hi(xb) >> 20) & 0xf0u);
    return s.x == b0 * off_top && s.y == b1 * off_top && s.z == b2 * off_top && s.w == b3 * off_top;
}

// One pass of 16 genes: CIP(t-1) (rule R1), QIP(t), the packed item sums; xbits holds the
// 16 alleles (the first vector's in bits 0-7). The fixed-allele test covers both vectors.
template <bool kCip>
__device__ __forceinline__ void qubit_pass2(const GenParams &p, const SegCtx2 &g, uint4 &s0, uint4 &s1,
                                            int32_t c, int32_t t, const unsigned char *thr_bytes,
                                            bool &fixed, int &countdown, uint32_t &xbits, uint32_t &accn)
{
    const uint32_t off_top = (uint32_t)(8 * p.K);
    const uint32_t k8 = off_top * 0x00010001u;
    accn = 0u;
    fixed = false;
    if (countdown == 0) {
        const int bp = __ffs((int)off_top) - 1;
        uint32_t xa0, xb0, xs0, xa1, xb1, xs1;
        const bool sat = saturated_vec(s0, off_top, bp, xa0, xb0, xs0) & saturated_vec(s1, off_top, bp, xa1, xb1, xs1);
        const bool ok = sat && (!kCip || (xs0 == g.e0 && xs1 == g.e1));
        if (__all_sync(0xffffffffu, ok)) {
            fixed = true;
            xbits = xs0 | (xs1 << 8);
            const uint4 ib = s_item_bytes[threadIdx.x], ib2 = s_item_bytes2[threadIdx.x];
            const uint32_t sw = __dp4a(xa0, ib.x, __dp4a(xb0, ib.y, __dp4a(xa1, ib2.x, __dp4a(xb1, ib2.y, 0u))));
            const uint32_t sv = __dp4a(xa0, ib.z, __dp4a(xb0, ib.w, __dp4a(xa1, ib2.z, __dp4a(xb1, ib2.w, 0u))));
            accn = sw | (sv << 16);
            return;
        }
        countdown = 15;
    } else {
        --countdown;
    }
    if (kCip) {
        const uint4 d = s_delta[threadIdx.x], d2 = s_delta2[threadIdx.x];
        s0.x = rotate_pair_signed(s0.x, d.x, k8);
        s0.y = rotate_pair_signed(s0.y, d.y, k8);
        s0.z = rotate_pair_signed(s0.z, d.z, k8);
        s0.w = rotate_pair_signed(s0.w, d.w, k8);
        s1.x = rotate_pair_signed(s1.x, d2.x, k8);
        s1.y = rotate_pair_signed(s1.y, d2.y, k8);
        s1.z = rotate_pair_signed(s1.z, d2.z, k8);
        s1.w = rotate_pair_signed(s1.w, d2.w, k8);
    }
    const uint32_t sp[8] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
    const Draw4 r0 = philox4x32_10_rk(g.ctr0, (uint32_t)c, (uint32_t)t, 0u, p.rk0, p.rk1);
    const Draw4 r1 = philox4x32_10_rk(g.ctr0 + 1u, (uint32_t)c, (uint32_t)t, 0u, p.rk0, p.rk1);
    const Draw4 r2 = philox4x32_10_rk(g.ctr0 + 2u, (uint32_t)c, (uint32_t)t, 0u, p.rk0, p.rk1);
    const Draw4 r3 = philox4x32_10_rk(g.ctr0 + 3u, (uint32_t)c, (uint32_t)t, 0u, p.rk0, p.rk1);
    const uint32_t u[16] = {r0.a, r0.b, r0.c, r0.d, r1.a, r1.b, r1.c, r1.d,
                            r2.a, r2.b, r2.c, r2.d, r3.a, r3.b, r3.c, r3.d};
    xbits = 0u;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const uint32_t off = (i & 1) ? (sp[i >> 1] >> 16) : (sp[i >> 1] & 0xffffu);
        const uint32_t thr = *reinterpret_cast<const uint32_t *>(thr_bytes + off);
        if ((u[i] < thr) || (off == off_top)) {
            xbits |= 1u << i;
            accn += g.wv[i];
        }
    }
}

// One tile segment (rows ra .. ra + seg_rows - 1 of tile `tile`) of one generation, 16
// genes per thread and pass, the state streamed through a per-thread cp.async ring of
// kRing2Stages slots of 32 bytes (ring: this block's ring; slot s, half h of thread i at
// ring[(2 s + h) * kThreads + i]).
template <bool kCip>
__device__ __forceinline__ void ring_segment2(const GenParams &p, int tile, int ra, int seg_rows, int32_t t,
                                              uint8_t *x_cur, const uint8_t *elite_row,
                                              const unsigned char *thr_bytes, uint4 *ring, uint32_t *s_acc32,
                                              int &countdown)
{
    SegCtx2 g;
    seg_setup2<kCip>(p, g, tile, elite_row);
    const int ra_key = ra + p.row0;
    const bool leader = (threadIdx.x & 31) == 0;
    uint4 *slots = ring + threadIdx.x;
    uint4 *sptr = p.state + (size_t)ra * p.svec + g.vec;
    const size_t sstep = (size_t)p.svec;
    uint8_t *xptr = x_cur + (size_t)ra * p.xstride + g.vec;
    const size_t xstep = (size_t)p.xstride;
    const uint4 *ld_ptr = sptr;
    uint4 *st_ptr = sptr;
    uint8_t *xst_ptr = xptr;
    auto issue = [&](uint32_t stage, bool v) {
        uint4 *dst = slots + (size_t)stage * 2 * kThreads;
        const bool v0 = v && g.act0, v1 = v && g.act1;
        cp_async16(dst, v0 ? (const void *)ld_ptr : (const void *)p.state, v0 ? 16u : 0u);
        cp_async16(dst + kThreads, v1 ? (const void *)(ld_ptr + 1) : (const void *)p.state, v1 ? 16u : 0u);
        cp_async_commit();
        ld_ptr += sstep;
    };
#pragma unroll
    for (int k = 0; k < kRing2Stages - 1; ++k) issue((uint32_t)k, k < seg_rows);
    const int lim = seg_rows - (kRing2Stages - 1);
    for (int pass = 0; pass < seg_rows; ++pass) {
        issue((uint32_t)(pass + kRing2Stages - 1) & (kRing2Stages - 1), pass < lim);
        cp_async_wait<kRing2Stages - 1>();
        const uint32_t slot = (uint32_t)pass & (kRing2Stages - 1);
        uint4 s0 = slots[(size_t)slot * 2 * kThreads];
        uint4 s1 = slots[(size_t)slot * 2 * kThreads + kThreads];
        uint32_t xbits, accn;
        bool fixed;
        qubit_pass2<kCip>(p, g, s0, s1, ra_key + pass, t, thr_bytes, fixed, countdown, xbits, accn);
        if (!fixed) {                   // a fixed pass leaves the state as it is
            if (g.act0) st_ptr[0] = s0;
            if (g.act1) st_ptr[1] = s1;
        }
        if (g.act1) *reinterpret_cast<uint16_t *>(xst_ptr) = (uint16_t)xbits;
        else if (g.act0) *xst_ptr = (uint8_t)xbits;
        add_row_sums<true>(32, leader, true, pass, accn, 0, 0, s_acc32, nullptr);
        st_ptr += sstep;
        xst_ptr += xstep;
    }
    cp_async_wait<0>();
    flush_segment<true>(p, t, ra, seg_rows, s_acc32, nullptr);
}

// ---------------------------------------------------------------------------------------
// Resident form: a cooperative run whose blocks keep their share of the state in shared
// memory for the whole run. A population whose state fits in the SMs' combined shared
// memory (about 34 MB on a GB300, e.g. 1,024 x 10,000 genes = 20 MB) is read from device
// memory once at the start of a run and written back once at its end; in between, a
// generation reads and writes nothing but the allele plane, the row sums and the elite key
// in device memory. Each block owns the same equal share of tile-rows in every generation
// (no queue: the share is fixed because its state lives in the block), and the blocks meet
// at the bounded grid barrier of the deferred close between generations.
// ---------------------------------------------------------------------------------------

// One segment (rows ra .. ra + seg_rows - 1 of tile `tile`) of one generation on the
// resident state st (thread (r_sub, v_in) of row rr at st[rr * tile_vecs + v_in]).
// g: the segment's items (seg_items, this tile) and elite alleles (seg_elite).
template <bool kNarrow, int kRule, bool kCip, bool kSegDelta>
__device__ __forceinline__ void resident_segment(const GenParams &p, const BlockShare &b, const SegCtx &g,
                                                 int ra, int seg_rows, int32_t t, const uint8_t *x_prev,
                                                 uint8_t *x_cur, const unsigned char *thr_bytes, uint4 *st,
                                                 uint32_t *s_acc32, unsigned long long *s_acc64,
                                                 int &countdown)
{
    const int rpp = b.rows_per_pass;
    const int passes = (seg_rows + rpp - 1) / rpp;
    const int ra_key = ra + p.row0;
    uint4 *sp = st + (size_t)b.r_sub * b.tile_vecs + b.v_in;
    const int sstep = rpp * b.tile_vecs;
    uint8_t *xptr = x_cur + ((size_t)ra + b.r_sub) * p.xstride + g.vec;
    const uint8_t *xoptr = x_prev + ((size_t)ra + b.r_sub) * p.xstride + g.vec;
    const size_t xstep = (size_t)rpp * p.xstride;
    int rr = b.r_sub;
    for (int pass = 0; pass < passes; ++pass) {
        const bool ok = rr < seg_rows;
        const bool live = g.active && ok;
        uint4 sv = live ? *sp : make_uint4(0, 0, 0, 0);
        const uint32_t xo = (kRule == 1 && kCip && live) ? (uint32_t)*xoptr : 0u;
        uint32_t xbits, accn;
        int64_t acw, acv;
        bool fixed;
        sv = qubit_pass<kNarrow, kRule, kCip, ParamKeys, kSegDelta>(p, ParamKeys{p}, g, sv, xo, ra_key + rr, t,
                                                                    thr_bytes, fixed, countdown, xbits, accn,
                                                                    acw, acv);
        if (live) {
            if (!fixed) *sp = sv;
            *xptr = (uint8_t)xbits;
        }
        add_row_sums<kNarrow>(b.lanes, b.leader, ok, rr, accn, acw, acv, s_acc32, s_acc64);
        sp += sstep;
        xptr += xstep;
        xoptr += xstep;
        rr += rpp;
    }
    flush_segment<kNarrow>(p, t, ra, seg_rows, s_acc32, s_acc64);
}

// Copies the block's share of the state between device memory and the resident copy
// (to_smem: at the start of a run; otherwise at its end), optionally applying the CIP of
// generation t toward elite row `elite` on the way out (the run's final rotation).
template <int kRule, bool kToSmem>
__device__ __forceinline__ void resident_copy(const GenParams &p, const BlockShare &b, uint4 *st,
                                              int32_t t, const uint8_t *elite)
{
    const int64_t n = (b.u_end - b.u_begin) * b.tile_vecs;
    const int sh = __ffs(b.tile_vecs) - 1;
    const uint8_t *xl = p.xbits + (size_t)(t & 1) * p.xplane;
    const uint32_t k8 = (uint32_t)(8 * p.K) * 0x00010001u;
    for (int64_t i = threadIdx.x; i < n; i += kThreads) {
        const int64_t u = b.u_begin + (i >> sh);
        const int tile = (int)(u / p.np);
        const int64_t row = u - (int64_t)tile * p.np;
        const int vec = tile * b.tile_vecs + (int)(i & (b.tile_vecs - 1));
        if (vec >= p.svec) continue;
        const size_t gi = (size_t)row * p.svec + vec;
        if constexpr (kToSmem) {
            st[i] = p.state[gi];
        } else {
            const uint32_t e8 = elite[vec];
            const uint32_t m8 = kRule == 1 ? (e8 ^ (uint32_t)xl[(size_t)row * p.xstride + vec]) : 0xffu;
            p.state[gi] = rotate_vec(st[i], e8, m8, k8);
        }
    }
}

// Records of generation t in a resident run (block 0, all threads): the best-so-far record
// is kept by thread 0 in registers for the whole run (no other block writes it), so writing
// a generation's records costs no read of device memory unless the best row changes.
__device__ __forceinline__ void record_resident(const GenParams &p, int32_t t, int32_t e, int64_t f,
                                                int64_t &best_f, int64_t &best_g)
{
    __shared__ int32_t s_improved;
    if (threadIdx.x == 0) {
        p.hist_e[t] = e;
        p.hist_f[t] = f;
        *p.elite_idx = e;
        const int improved = (best_g < 0 || f > best_f) ? 1 : 0;
        if (improved) {
            best_f = f;
            best_g = t;
            p.best[0] = f;
            p.best[1] = t;
            p.best[2] = e;
        }
        s_improved = improved;
    }
    __syncthreads();
    if (s_improved) {
        const uint4 *src = reinterpret_cast<const uint4 *>(
            p.xbits + (size_t)(t & 1) * p.xplane + (size_t)e * p.xstride);
        uint4 *dst = reinterpret_cast<uint4 *>(p.best_row);
        for (int i = threadIdx.x; i < p.xstride / 16; i += kThreads) dst[i] = __ldcg(src + i);
    }
}

// Dynamic shared memory: [resident state: share_max tile-rows x tile_vecs uint4][row sums].
template <bool kNarrow, int kRule, bool kSegDelta>
__global__ void __launch_bounds__(kThreads, kNarrow ? 3 : 2) resident_run_kernel(const GenParams p, int32_t G,
                                                                                  int32_t share_max)
{
    __shared__ uint32_t s_thr[kMaxThr];
    __shared__ int s_e;
    __shared__ long long s_f;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    load_thresholds(p, s_thr);
    grid_dependency_wait();
    const BlockShare b = block_share(p);
    uint4 *st = reinterpret_cast<uint4 *>(smem_raw);
    unsigned char *acc = smem_raw + (size_t)share_max * b.tile_vecs * sizeof(uint4);
    uint32_t *s_acc32 = reinterpret_cast<uint32_t *>(acc);
    unsigned long long *s_acc64 = reinterpret_cast<unsigned long long *>(acc);
    const unsigned char *thr_bytes = reinterpret_cast<const unsigned char *>(s_thr);
    const int32_t t0 = *p.gen;
    resident_copy<kRule, true>(p, b, st, t0, nullptr);
    clear_row_sums<kNarrow>(p.seg_rows_max, s_acc32, s_acc64);   // (its barrier orders the copy)
    int countdown = 0;
    int32_t e = 0;
    int64_t best_f = 0, best_g = -1;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        best_f = __ldcg(p.best);
        best_g = __ldcg(p.best + 1);
    }
    const bool stamp = p.gen_ns != nullptr && blockIdx.x == 0 && threadIdx.x == 0;
    if (stamp) p.gen_ns[0] = global_ns();
    for (int32_t g = 0; g <= G; ++g) {
        const int32_t t = t0 + g;
        int64_t f = 0;
        if (g > 0) {
            if (!grid_wait<true>(p, (unsigned int)g * gridDim.x)) return;
            if (stamp) p.gen_ns[g] = global_ns();
            if (threadIdx.x == 0) {
                int32_t ee;
                int64_t ff;
                elite_from_key(p, t - 1, ee, ff);
                s_e = ee;
                s_f = ff;
            }
            __syncthreads();
            e = s_e;
            f = s_f;
            if (blockIdx.x == 0) record_resident(p, t - 1, e, f, best_f, best_g);
        }
        if (g == G) break;
        if (blockIdx.x == 0 && threadIdx.x == 0) *key_slot(p, t + 1) = 0ull;
        const uint8_t *x_prev = p.xbits + (size_t)((t + 1) & 1) * p.xplane;
        uint8_t *x_cur = p.xbits + (size_t)(t & 1) * p.xplane;
        const uint8_t *elite_row = x_prev + (size_t)e * p.xstride;
        for (int64_t u0 = b.u_begin; u0 < b.u_end;) {
            const int tile = (int)(u0 / p.np);
            const int ra = (int)(u0 - (int64_t)tile * p.np);
            const int seg_rows = (int)min(min((int64_t)(p.np - ra), b.u_end - u0), (int64_t)p.seg_rows_max);
            uint4 *seg_st = st + (size_t)(u0 - b.u_begin) * b.tile_vecs;
            SegCtx sg;
            seg_items<kNarrow>(p, sg, tile, b.v_in, b.tile_vecs);
            if (g == 0) {
                resident_segment<kNarrow, kRule, false, kSegDelta>(p, b, sg, ra, seg_rows, t, x_prev, x_cur,
                                                                   thr_bytes, seg_st, s_acc32, s_acc64, countdown);
            } else {
                seg_elite<true, kSegDelta>(sg, elite_row);
                resident_segment<kNarrow, kRule, true, kSegDelta>(p, b, sg, ra, seg_rows, t, x_prev, x_cur,
                                                                  thr_bytes, seg_st, s_acc32, s_acc64, countdown);
            }
            u0 += seg_rows;
        }
        grid_arrive(p);
    }
    // the run's final CIP on the way back to device memory
    const int32_t t_last = t0 + G - 1;
    resident_copy<kRule, false>(p, b, st, t_last,
                                p.xbits + (size_t)(t_last & 1) * p.xplane + (size_t)e * p.xstride);
}

// ---------------------------------------------------------------------------------------
// generation_kernel: one generation per launch.
//
// Deferred close (device DetermineElite with the packed elite key, the default): no block
// waits for another. Every block reads the elite of generation t - 1 from its key slot at
// its start (the previous launch has completed, so every row of t - 1 is in the key) and
// rotates toward it; block 0 also writes the records of t - 1 and clears the key slot of
// t + 1. The records of a run's last generation are written by the final CIP launch, and a
// last one-thread launch advances the generation counter by the run. The convergence test
// of generation t - 1 is evaluated by every block from the same data (the key of t - 1,
// the run length and elite fitness recorded for t - 2), so all blocks agree; when it holds,
// the launch applies the CIP of t - 1 alone and block 0 marks the instance stopped.
//
// Otherwise (elite by a scan of fitness[] when the fitness does not fit the key, or the
// host DetermineElite variant): the last block to finish closes the generation.
// ---------------------------------------------------------------------------------------
// Three blocks per SM (the host's grid), so up to 85 registers a thread: the compiler takes
// 76 for the narrow ring form, which measured c3 348 vs 361 us per generation against the
// 64 that four blocks would allow.
//
// kF: the variant for instances that keep F (packed sums, 16-bit state, the ring, deferred
// close with a segment queue; rule R1 with per-segment deltas, or R2); the host runs it only
// so.
template <bool kNarrow, int kRule, bool kRing, bool kS8 = false, bool kSegDelta = false, bool kF = false>
__global__ void __launch_bounds__(kThreads, kNarrow ? 3 : 2) generation_kernel(const GenParams p)
{
    __shared__ uint32_t s_thr[kMaxThr];
    __shared__ int s_last, s_stop, s_t, s_e;
    __shared__ long long s_f;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    SmemParts m = carve_smem<kRing>(smem_raw);
    load_thresholds(p, s_thr);
    grid_dependency_wait();
    if (p.deferred) {
        if (threadIdx.x == 0) {
            const int32_t t = *p.gen + p.g;
            int stop = deferred_skip(p, t) ? kStopped : kRunning;
            int32_t e = 0;
            int64_t f = 0;
            if (stop == kRunning && p.apply_cip) {
                elite_from_key(p, t - 1, e, f);
                if (p.converge) {   // did generation t - 1 meet the convergence test?
                    const int32_t prev = t - 1 > 0 ? p.conv[(t - 2) & 1] : 0;
                    const int32_t run = (prev > 0 && f == p.hist_f[t - 2]) ? prev + 1 : 1;
                    if (run >= kConvergeWindow) stop = kStopPending;
                }
            }
            s_t = t;
            s_stop = stop;
            s_e = e;
            s_f = f;
        }
        __syncthreads();
        const int32_t stop = s_stop, t = s_t, e_prev = s_e;
        const int64_t f_prev = s_f;
        if (stop == kStopped) return;
        const BlockShare b = block_share(p);
        if (blockIdx.x == 0) {
            if (p.apply_cip) {
                record_generation(p, t - 1, e_prev, f_prev);
                if (stop == kStopPending && threadIdx.x == 0) {
                    p.conv[3] = t - 1;
                    __threadfence();
                    st_release(p.conv + 2, kStopped);
                }
            }
            if (threadIdx.x == 0) {
                *key_slot(p, t + 1) = 0ull;
                p.qctr[(t + 1) % 3] = 0u;
                if (kF) {
                    p.fcnt[(t + 1) % 3] = 0ull;
                    p.fcnt[4 + (t + 1) % 3] = 0ull;
                    if (t >= 1 && p.hist_d) p.hist_d[t - 1] = p.fcnt[4 + (t + 2) % 3];
                }
            }
        }
        if (stop == kStopPending) {
            final_cip_body<kRule, kS8>(p, b, t - 1, e_prev);   // the CIP of the converged generation
            return;
        }
        if (p.apply_cip)
            one_generation<kNarrow, kRule, true, kRing, kS8, kSegDelta, kF>(p, b, t, e_prev, m, s_thr, true);
        else
            one_generation<kNarrow, kRule, false, kRing, kS8, kSegDelta, kF>(p, b, t, e_prev, m, s_thr, true);
        allow_dependent_launch();
        return;
    }

    if (threadIdx.x == 0) s_stop = stop_state(p);
    __syncthreads();
    const int32_t stop = s_stop;
    if (stop == kStopped) return;            // converged in an earlier launch
    const BlockShare b = block_share(p);
    const int32_t t = *p.gen;
    const int32_t e_prev = *p.elite_idx;
    if (stop == kStopPending) {
        // the generation before met the convergence test: its CIP alone, then stopped
        final_cip_body<kRule, kS8>(p, b, t - 1, e_prev);
    } else if (p.apply_cip) {
        one_generation<kNarrow, kRule, true, kRing, kS8>(p, b, t, e_prev, m, s_thr);
    } else {
        one_generation<kNarrow, kRule, false, kRing, kS8>(p, b, t, e_prev, m, s_thr);
    }

    // The next generation's blocks may start their prologue now.
    allow_dependent_launch();
    if (!p.do_de && stop == kRunning) return;
    // Ticket: the barrier orders every thread's writes of this block before thread 0's
    // release; the last block's acquire (then its barrier) makes all blocks' writes visible
    // to the close.
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int prev = atom_add_acq_rel(p.ticket, 1u);
        s_last = (prev == gridDim.x - 1u) ? 1 : 0;
    }
    __syncthreads();
    if (!s_last) return;
    if (stop == kStopPending) {
        if (threadIdx.x == 0) {
            *p.ticket = 0u;
            p.conv[2] = kStopped;
        }
        return;
    }
    close_generation(p, t);
    if (threadIdx.x == 0) {
        *p.gen = t + 1;
        *p.ticket = 0u;
        *p.bar_gen = t + 1;
    }
}

// End of a deferred-close run of G generations: advances the generation counter (to one past
// the generation that met the convergence test, if the instance stopped) and clears the
// three key slots and segment-queue counters. One thread.
__global__ void end_run_kernel(const GenParams p, int32_t G)
{
    grid_dependency_wait();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int32_t gen = *p.gen;
    int32_t next = gen + G;
    if (p.converge && p.conv[2] == kStopped) next = min(next, p.conv[3] + 1);
    *p.gen = next;
    *p.bar_gen = next;
    *p.ticket = 0u;   // the arrival counter of a cooperative run
    p.keys[0] = p.keys[1] = p.keys[2] = 0ull;
    p.qctr[0] = p.qctr[1] = p.qctr[2] = 0u;
}

// Records of a generation whose elite e was picked on the host (host DetermineElite).
__global__ void __launch_bounds__(kThreads) record_elite_kernel(const GenParams p, int32_t e)
{
    __shared__ int s_improved;
    const int tid = threadIdx.x;
    grid_dependency_wait();
    const int32_t t = *p.gen;
    if (tid == 0) {
        const int64_t fe = p.fitness[e];
        p.hist_e[t] = e;
        p.hist_f[t] = fe;
        *p.elite_idx = e;
        *key_slot(p, t) = 0ull;
        const int improved = (p.best[1] < 0 || fe > p.best[0]) ? 1 : 0;
        if (improved) {
            p.best[0] = fe;
            p.best[1] = t;
            p.best[2] = e;
        }
        s_improved = improved;
    }
    __syncthreads();
    if (s_improved) {
        const uint4 *src = reinterpret_cast<const uint4 *>(
            p.xbits + (size_t)(t & 1) * p.xplane + (size_t)e * p.xstride);
        for (int i = tid; i < p.xstride / 16; i += kThreads)
            reinterpret_cast<uint4 *>(p.best_row)[i] = src[i];
    }
    if (tid == 0) {
        *p.gen = t + 1;
        *p.bar_gen = t + 1;
    }
}

// CIP of the last generation of a run launched generation by generation.
// CIP toward elite e of generation t over the whole state (grid-stride), 16-bit or byte
// storage.
template <int kRule, bool kS8>
__device__ __forceinline__ void rotate_toward(const GenParams &p, int32_t t, const uint8_t *elite)
{
    const uint8_t *xl = p.xbits + (size_t)(t & 1) * p.xplane;
    const uint32_t k8 = (uint32_t)(8 * p.K) * 0x00010001u;
    const size_t total = (size_t)p.np * p.svec;
    for (size_t i = (size_t)blockIdx.x * kThreads + threadIdx.x; i < total;
         i += (size_t)gridDim.x * kThreads) {
        const size_t c = i / (size_t)p.svec;
        const size_t v = i - c * (size_t)p.svec;
        const uint32_t e8 = elite[v];
        const uint32_t m8 = kRule == 1 ? (e8 ^ (uint32_t)xl[c * p.xstride + v]) : 0xffu;
        if constexpr (kS8) {
            uint2 *s8 = reinterpret_cast<uint2 *>(p.state) + i;
            *s8 = pack8(rotate_vec(unpack8(*s8), e8, m8, k8));
        } else {
            p.state[i] = rotate_vec(p.state[i], e8, m8, k8);
        }
    }
}

template <int kRule, bool kS8>
__device__ __forceinline__ void rotate_all(const GenParams &p, int32_t t, int32_t e)
{
    rotate_toward<kRule, kS8>(p, t, p.xbits + (size_t)(t & 1) * p.xplane + (size_t)e * p.xstride);
}

// CIP of generation t of a row block toward an elite row supplied from outside (packed
// alleles, bit i of byte v = gene 8v + i): the rotation step of a population sharded by
// rows, whose elite may live in another block.
template <int kRule>
__global__ void __launch_bounds__(kThreads) rows_cip_kernel(const GenParams p, int32_t t, const uint8_t *elite)
{
    if (p.state8) rotate_toward<kRule, true>(p, t, elite);
    else rotate_toward<kRule, false>(p, t, elite);
}

template <int kRule>
__global__ void __launch_bounds__(kThreads) cip_kernel(const GenParams p)
{
    __shared__ int s_stop, s_last, s_t, s_e;
    __shared__ long long s_f;
    grid_dependency_wait();
    if (p.deferred) {
        // the final CIP of a deferred-close run of p.g generations: elite of the last
        // generation from its key; block 0 writes that generation's records
        if (threadIdx.x == 0) {
            const int32_t t_last = *p.gen + p.g - 1;
            const int skip = deferred_skip(p, t_last + 1);
            int32_t e = 0;
            int64_t f = 0;
            if (!skip) elite_from_key(p, t_last, e, f);
            s_stop = skip;
            s_t = t_last;
            s_e = e;
            s_f = f;
        }
        __syncthreads();
        if (s_stop) return;
        const int32_t t_last = s_t, e = s_e;
        if (blockIdx.x == 0) {
            if (threadIdx.x == 0 && p.fword && p.hist_d) p.hist_d[t_last] = p.fcnt[4 + t_last % 3];
            const int32_t run = record_generation(p, t_last, e, s_f);
            if (run >= kConvergeWindow && threadIdx.x == 0) {
                p.conv[3] = t_last;
                __threadfence();
                st_release(p.conv + 2, kStopped);
            }
        }
        if (p.state8) rotate_all<kRule, true>(p, t_last, e);
        else rotate_all<kRule, false>(p, t_last, e);
        return;
    }
    if (threadIdx.x == 0) s_stop = stop_state(p);
    __syncthreads();
    const int32_t stop = s_stop;
    if (stop == kStopped) return;
    const int32_t t_last = *p.gen - 1;
    const int32_t e = *p.elite_idx;
    if (p.state8) rotate_all<kRule, true>(p, t_last, e);
    else rotate_all<kRule, false>(p, t_last, e);
    if (stop == kStopPending) {   // the run's last generation met the convergence test
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) s_last = atomicAdd(p.ticket, 1u) == gridDim.x - 1u ? 1 : 0;
        __syncthreads();
        if (s_last && threadIdx.x == 0) {
            *p.ticket = 0u;
            p.conv[2] = kStopped;
        }
    }
}

// generation_kernel2: the deferred-close generation launch with 16 genes per thread and
// pass (ring_segment2; rule R1, packed items <= 127, 16-bit state). p describes tiles of 512
// vectors (ntile, units, the segment queue); dynamic shared memory: the ring
// (kRing2Stages x 2 x kThreads x 16 B), then the row sums of a segment.
template <bool kCip>
__device__ __forceinline__ void generation2_body(const GenParams &p, int32_t t, int32_t e_prev,
                                                 unsigned char *smem, const uint32_t *s_thr)
{
    __shared__ int32_t s_qi;
    uint4 *ring = reinterpret_cast<uint4 *>(smem);
    uint32_t *s_acc32 = reinterpret_cast<uint32_t *>(smem + (size_t)kRing2Stages * 2 * kThreads * 16);
    const unsigned char *thr_bytes = reinterpret_cast<const unsigned char *>(s_thr);
    const uint8_t *x_prev = p.xbits + (size_t)((t + 1) & 1) * p.xplane;
    uint8_t *x_cur = p.xbits + (size_t)(t & 1) * p.xplane;
    const uint8_t *elite_row = x_prev + (size_t)e_prev * p.xstride;
    int countdown = 0;
    clear_row_sums<true>(p.seg_rows_max, s_acc32, nullptr);
    if (p.nsegs > 0) {
        unsigned int *ctr = p.qctr + (t % 3);
        for (;;) {
            if (threadIdx.x == 0) s_qi = (int32_t)atomicAdd(ctr, 1u);
            __syncthreads();
            const int32_t qi = s_qi;
            if (qi >= p.nsegs) break;
            const int4 sg = __ldg(p.segq + qi);
            ring_segment2<kCip>(p, sg.x, sg.y, sg.z, t, x_cur, elite_row, thr_bytes, ring, s_acc32, countdown);
        }
    } else {
        const BlockShare b = block_share(p);
        for (int64_t u0 = b.u_begin; u0 < b.u_end;) {
            const int tile = (int)(u0 / p.np);
            const int ra = (int)(u0 - (int64_t)tile * p.np);
            const int seg_rows = (int)min(min((int64_t)(p.np - ra), b.u_end - u0), (int64_t)p.seg_rows_max);
            u0 += seg_rows;
            ring_segment2<kCip>(p, tile, ra, seg_rows, t, x_cur, elite_row, thr_bytes, ring, s_acc32, countdown);
        }
    }
}

__global__ void __launch_bounds__(kThreads, 2) generation_kernel2(const GenParams p)
{
    __shared__ uint32_t s_thr[kMaxThr];
    __shared__ int s_stop, s_t, s_e;
    __shared__ long long s_f;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    load_thresholds(p, s_thr);
    grid_dependency_wait();
    if (threadIdx.x == 0) {
        const int32_t t = *p.gen + p.g;
        int stop = deferred_skip(p, t) ? kStopped : kRunning;
        int32_t e = 0;
        int64_t f = 0;
        if (stop == kRunning && p.apply_cip) {
            elite_from_key(p, t - 1, e, f);
            if (p.converge) {
                const int32_t prev = t - 1 > 0 ? p.conv[(t - 2) & 1] : 0;
                const int32_t run = (prev > 0 && f == p.hist_f[t - 2]) ? prev + 1 : 1;
                if (run >= kConvergeWindow) stop = kStopPending;
            }
        }
        s_t = t;
        s_stop = stop;
        s_e = e;
        s_f = f;
    }
    __syncthreads();
    const int32_t stop = s_stop, t = s_t, e_prev = s_e;
    const int64_t f_prev = s_f;
    if (stop == kStopped) return;
    if (blockIdx.x == 0) {
        if (p.apply_cip) {
            record_generation(p, t - 1, e_prev, f_prev);
            if (stop == kStopPending && threadIdx.x == 0) {
                p.conv[3] = t - 1;
                __threadfence();
                st_release(p.conv + 2, kStopped);
            }
        }
        if (threadIdx.x == 0) {
            *key_slot(p, t + 1) = 0ull;
            p.qctr[(t + 1) % 3] = 0u;
        }
    }
    if (stop == kStopPending) {
        // the CIP of the converged generation (grid-stride over the whole state)
        if (p.state8) rotate_all<0, true>(p, t - 1, e_prev);
        else rotate_all<0, false>(p, t - 1, e_prev);
        return;
    }
    if (p.apply_cip) generation2_body<true>(p, t, e_prev, smem_raw, s_thr);
    else generation2_body<false>(p, t, e_prev, smem_raw, s_thr);
    allow_dependent_launch();
}

// ---------------------------------------------------------------------------------------
// Unfused form: the four steps of a generation as four launches, the way the paper offloads
// them as separate target regions (Sec. III-B): cip_kernel (CIP toward the previous elite),
// qip_kernel (observation of every qubit into the allele plane), eval_kernel (eq. (1) per
// chromosome from the alleles) and de_kernel (DetermineElite and the records). Each step
// passes its result to the next through device memory, so the state is read twice and
// written once per generation and the alleles are written once and read once; the results
// equal the fused kernel's.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) qip_kernel(const GenParams p)
{
    __shared__ uint32_t s_thr[kMaxThr];
    load_thresholds(p, s_thr);
    __syncthreads();
    const unsigned char *thr_bytes = reinterpret_cast<const unsigned char *>(s_thr);
    const int32_t t = *p.gen;
    uint8_t *x_cur = p.xbits + (size_t)(t & 1) * p.xplane;
    const uint32_t off_top = (uint32_t)(8 * p.K);
    const size_t total = (size_t)p.np * p.svec;
    for (size_t i = (size_t)blockIdx.x * kThreads + threadIdx.x; i < total;
         i += (size_t)gridDim.x * kThreads) {
        const size_t c = i / (size_t)p.svec;
        const size_t v = i - c * (size_t)p.svec;
        const uint4 s = p.state[i];
        const uint32_t sp[4] = {s.x, s.y, s.z, s.w};
        const uint32_t ck = (uint32_t)c + (uint32_t)p.row0;
        const Draw4 r0 = philox4x32_10_rk(2u * (uint32_t)v, ck, (uint32_t)t, 0u, p.rk0, p.rk1);
        const Draw4 r1 = philox4x32_10_rk(2u * (uint32_t)v + 1u, ck, (uint32_t)t, 0u, p.rk0, p.rk1);
        const uint32_t u[8] = {r0.a, r0.b, r0.c, r0.d, r1.a, r1.b, r1.c, r1.d};
        uint32_t xbits = 0u;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint32_t off = (k & 1) ? (sp[k >> 1] >> 16) : (sp[k >> 1] & 0xffffu);
            const uint32_t thr = *reinterpret_cast<const uint32_t *>(thr_bytes + off);
            if ((u[k] < thr) || (off == off_top)) xbits |= 1u << k;
        }
        x_cur[c * p.xstride + v] = (uint8_t)xbits;
    }
}

// Row sums of one chromosome per block iteration from its alleles and the 32-bit items
// (zero on the padding genes), then eq. (1) into fitness[c].
__global__ void __launch_bounds__(kThreads) eval_kernel(const GenParams p)
{
    __shared__ long long s_w[kThreads / 32], s_v[kThreads / 32];
    const int32_t t = *p.gen;
    const uint8_t *x_cur = p.xbits + (size_t)(t & 1) * p.xplane;
    for (int32_t c = blockIdx.x; c < p.np; c += gridDim.x) {
        const uint8_t *xr = x_cur + (size_t)c * p.xstride;
        long long w = 0, v = 0;
        for (int32_t vec = threadIdx.x; vec < p.svec; vec += kThreads) {
            const uint32_t xb = xr[vec];
            if (!xb) continue;
            const int4 a = __ldg(p.w4 + 2 * (size_t)vec), b = __ldg(p.w4 + 2 * (size_t)vec + 1);
            const int4 d = __ldg(p.v4 + 2 * (size_t)vec), e = __ldg(p.v4 + 2 * (size_t)vec + 1);
            const int32_t wi[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
            const int32_t vi[8] = {d.x, d.y, d.z, d.w, e.x, e.y, e.z, e.w};
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if ((xb >> k) & 1u) {
                    w += wi[k];
                    v += vi[k];
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            w += __shfl_xor_sync(0xffffffffu, w, o);
            v += __shfl_xor_sync(0xffffffffu, v, o);
        }
        if ((threadIdx.x & 31) == 0) {
            s_w[threadIdx.x >> 5] = w;
            s_v[threadIdx.x >> 5] = v;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            long long sw = 0, sv = 0;
            for (int i = 0; i < kThreads / 32; ++i) {
                sw += s_w[i];
                sv += s_v[i];
            }
            p.fitness[c] = sw <= p.capacity ? (int64_t)sv : -p.lambda * ((int64_t)sw - p.capacity);
        }
        __syncthreads();
    }
}

// DetermineElite over fitness[] (lowest index of the maximum) and the records; one block.
__global__ void __launch_bounds__(kThreads) de_kernel(GenParams p)
{
    p.key_mode = 0;
    const int32_t t = *p.gen;
    close_generation(p, t);
    if (threadIdx.x == 0) {
        *p.gen = t + 1;
        *p.bar_gen = t + 1;
    }
}

// CIP with elite e of generation t_prev on one segment (one tile, rows ra .. ra + rows).
template <int kRule>
__device__ __forceinline__ void rotate_segment(const GenParams &p, const BlockShare &b, int tile, int ra,
                                               int rows, int32_t t_prev, int32_t e)
{
    const uint8_t *xl = p.xbits + (size_t)(t_prev & 1) * p.xplane;
    const int vec = tile * b.tile_vecs + b.v_in;
    if (vec >= p.svec) return;
    const uint32_t e8 = __ldcg(xl + (size_t)e * p.xstride + vec);
    const uint32_t k8 = (uint32_t)(8 * p.K) * 0x00010001u;
    for (int rr = b.r_sub; rr < rows; rr += b.rows_per_pass) {
        const size_t c = (size_t)ra + rr;
        const uint32_t m8 = kRule == 1 ? (e8 ^ (uint32_t)xl[c * p.xstride + vec]) : 0xffu;
        uint4 *sp = p.state + c * p.svec + vec;
        *sp = rotate_vec(*sp, e8, m8, k8);
    }
}

// ---------------------------------------------------------------------------------------
// Batched form: many independent instances in one persistent launch per generation. The
// host cuts every instance's ntile * np tile-rows into segments (one tile, at most
// kMaxSegRows rows each) of a few per block on average, ordered largest first; blocks take
// them from a queue. A block switches instance between segments (parameters, threshold
// table, tile geometry); each instance's ticket counts its finished segments, and the
// block that finishes an instance's last segment closes that instance's generation.
// Instances of one launch share the item-sum form and the rotation rule (the host groups
// them).
// ---------------------------------------------------------------------------------------
struct BatchSeg {
    int32_t inst, tile, ra, rows;
};

struct BatchArgs {
    const GenParams *params;      // [n] per-instance parameters
    const BatchSeg *segs;         // [nsegs] segments, largest first
    const int32_t *inst_segs;     // [n] segments per instance
    unsigned int *queue;          // [2] next segment to take, blocks finished (both 0
                                  // between launches: the last block clears them)
    unsigned int *done;           // [n] persistent form: generations of the run each
                                  // instance has closed (0 at the start of a run)
    int32_t nsegs;
    int32_t seg_rows_max;
};

template <bool kNarrow, int kRule, bool kCip>
__global__ void __launch_bounds__(kThreads, kNarrow ? 4 : 2) batch_generation_kernel(const BatchArgs a)
{
    __shared__ uint32_t s_thr[kMaxThr];
    __shared__ int s_last;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    SmemParts m = carve_smem<true>(smem_raw);
    const unsigned char *thr_bytes = reinterpret_cast<const unsigned char *>(s_thr);
    uint4 *slots = m.ring + threadIdx.x;
    __shared__ int32_t s_si, s_stop;
    grid_dependency_wait();
    clear_row_sums<kNarrow>(a.seg_rows_max, m.acc32, m.acc64);
    int countdown = 0;
    int32_t cur_inst = -1;
    int32_t table_K = -1;
    // Segments are taken from a shared queue in order (largest first), so blocks that draw
    // cheap segments (saturated instances, small rows) take more of them. The index is
    // read by every thread before the segment's first barrier, after which thread 0 may
    // overwrite it.
    for (;;) {
        if (threadIdx.x == 0) s_si = (int32_t)atomicAdd(a.queue, 1u);
        __syncthreads();
        const int32_t si = s_si;
        if (si >= a.nsegs) break;
        const BatchSeg sg = a.segs[si];
        const GenParams &p = a.params[sg.inst];
        if (sg.inst != cur_inst) {
            cur_inst = sg.inst;
            if (p.K != table_K) {           // table of this instance's D (row sums are clear)
                table_K = p.K;
                for (int i = threadIdx.x; i < 2 * p.K + 1; i += kThreads) s_thr[i] = p.thr[i];
                __syncthreads();
            }
        }
        if (threadIdx.x == 0) s_stop = stop_state(p);
        __syncthreads();
        const int32_t stop = s_stop;
        if (stop == kStopped) continue;      // converged earlier: no work, no ticket
        const int32_t t = *p.gen;
        const int32_t e_prev = *p.elite_idx;
        const uint8_t *x_prev = p.xbits + (size_t)((t + 1) & 1) * p.xplane;
        uint8_t *x_cur = p.xbits + (size_t)(t & 1) * p.xplane;
        const BlockShare b = tile_geometry(p.lanes, p.warps);
        if (stop == kStopPending)            // the CIP of the generation that converged
            rotate_segment<kRule>(p, b, sg.tile, sg.ra, sg.rows, t - 1, e_prev);
        else
            ring_segment<kNarrow, kRule, kCip, InlineKeys, false, false, true>(
                p, InlineKeys{p.rk0[0], p.rk1[0]}, b, sg.tile, sg.ra, sg.rows, t, x_prev, x_cur,
                x_prev + (size_t)e_prev * p.xstride, thr_bytes, slots, m.acc32, m.acc64, countdown);
        // the block that finishes an instance's last segment closes its generation (barrier
        // + release by thread 0, acquire by the last block's thread 0 + barrier)
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned int prev = atom_add_acq_rel(p.ticket, 1u);
            s_last = (prev == (unsigned int)a.inst_segs[sg.inst] - 1u) ? 1 : 0;
        }
        __syncthreads();
        if (s_last) {
            if (stop == kStopPending) {
                if (threadIdx.x == 0) {
                    *p.ticket = 0u;
                    p.conv[2] = kStopped;
                }
            } else {
                close_generation(p, t);
                if (threadIdx.x == 0) {
                    *p.gen = t + 1;
                    *p.ticket = 0u;
                    *p.bar_gen = t + 1;
                }
            }
            __syncthreads();
        }
    }
    allow_dependent_launch();
    // The last block to finish clears the queue for the next launch (which reads it only
    // after this grid has completed).
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(a.queue + 1, 1u) == gridDim.x - 1u) {
            a.queue[0] = 0u;
            a.queue[1] = 0u;
        }
    }
}

// Persistent form of a batched run: generations 2 .. G of the run (the first, which applies
// no CIP, is one batch_generation_kernel launch before it) in one cooperative launch. The
// work items are (step g, segment) in one queue over the launch, step-major with each step's
// segments largest first; a block takes the next item with one atomic. Before computing a
// segment of step g >= 1 of instance i the block waits (bounded, like the grid barrier of
// run_kernel) until instance i has closed its generation of step g - 1, which the block that
// finished that generation's last segment announces in done[i]. There is no grid-wide
// barrier: while the last segments of one instance's generation run, blocks already work on
// other instances' next generation. Items are taken in queue order and every block of the
// grid is resident (cooperative launch), so the earliest unfinished item never waits on a
// later one. Members with the convergence test use the per-generation form.
template <bool kNarrow, int kRule>
__global__ void __launch_bounds__(kThreads, kNarrow ? 4 : 2) batch_run_kernel(const BatchArgs a, int32_t G)
{
    __shared__ uint32_t s_thr[kMaxThr];
    __shared__ int s_last, s_ok;
    __shared__ uint32_t s_q;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    SmemParts m = carve_smem<true>(smem_raw);
    const unsigned char *thr_bytes = reinterpret_cast<const unsigned char *>(s_thr);
    uint4 *slots = m.ring + threadIdx.x;
    grid_dependency_wait();
    clear_row_sums<kNarrow>(a.seg_rows_max, m.acc32, m.acc64);
    int countdown = 0;
    int32_t table_K = -1;
    const uint32_t total = (uint32_t)G * (uint32_t)a.nsegs;
    for (;;) {
        if (threadIdx.x == 0) s_q = atomicAdd(a.queue, 1u);
        __syncthreads();
        const uint32_t q = s_q;
        if (q >= total) break;
        const int32_t step = (int32_t)(q / (uint32_t)a.nsegs);
        const BatchSeg sg = a.segs[q - (uint32_t)step * (uint32_t)a.nsegs];
        const GenParams &p = a.params[sg.inst];
        if (p.K != table_K) {               // table of this instance's D (row sums are clear)
            table_K = p.K;
            for (int i = threadIdx.x; i < 2 * p.K + 1; i += kThreads) s_thr[i] = p.thr[i];
        }
        if (threadIdx.x == 0) {
            int ok = 1;
            if (step > 0) {                 // the instance's previous generation must be closed
                const int32_t *dw = reinterpret_cast<const int32_t *>(a.done + sg.inst);
                const uint64_t deadline = global_ns() + p.wait_ns;
                ok = 0;
                for (uint32_t it = 0; it < (1u << 30); ++it) {
                    if (ld_acquire(dw) >= step) {
                        ok = 1;
                        break;
                    }
                    if (ld_acquire(p.error) != 0 || global_ns() > deadline) break;
                }
                if (!ok) atomicOr(p.error, kErrBarrierTimeout);
            }
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) continue;                // reported through the instance's error word
        const int32_t t = __ldcg(p.gen);
        const int32_t e_prev = __ldcg(p.elite_idx);
        const uint8_t *x_prev = p.xbits + (size_t)((t + 1) & 1) * p.xplane;
        uint8_t *x_cur = p.xbits + (size_t)(t & 1) * p.xplane;
        const BlockShare b = tile_geometry(p.lanes, p.warps);
        ring_segment<kNarrow, kRule, true, InlineKeys, false, false, true>(
            p, InlineKeys{p.rk0[0], p.rk1[0]}, b, sg.tile, sg.ra, sg.rows, t, x_prev, x_cur,
            x_prev + (size_t)e_prev * p.xstride, thr_bytes, slots, m.acc32, m.acc64, countdown);
        // the block that finishes the generation's last segment closes it and announces it
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned int prev = atom_add_acq_rel(p.ticket, 1u);
            s_last = (prev == (unsigned int)a.inst_segs[sg.inst] - 1u) ? 1 : 0;
        }
        __syncthreads();
        if (s_last) {
            close_generation(p, t);
            if (threadIdx.x == 0) {
                *p.gen = t + 1;
                *p.ticket = 0u;
                *p.bar_gen = t + 1;
                __threadfence();
                st_release(reinterpret_cast<int32_t *>(a.done + sg.inst), step + 1);
            }
            __syncthreads();
        }
    }
    // The last block to finish clears the queue for the next run.
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(a.queue + 1, 1u) == gridDim.x - 1u) {
            a.queue[0] = 0u;
            a.queue[1] = 0u;
        }
    }
}

// Final rotation of a batched run over the same segments (an instance that met the
// convergence test in the run's last generation is marked stopped by the block that
// rotates its last segment).
template <int kRule>
__global__ void __launch_bounds__(kThreads) batch_cip_kernel(const BatchArgs a)
{
    __shared__ int s_stop, s_last;
    grid_dependency_wait();
    for (int32_t si = blockIdx.x; si < a.nsegs; si += gridDim.x) {
        const BatchSeg sg = a.segs[si];
        const GenParams &p = a.params[sg.inst];
        __syncthreads();
        if (threadIdx.x == 0) s_stop = stop_state(p);
        __syncthreads();
        const int32_t stop = s_stop;
        if (stop == kStopped) continue;
        const BlockShare b = tile_geometry(p.lanes, p.warps);
        rotate_segment<kRule>(p, b, sg.tile, sg.ra, sg.rows, *p.gen - 1, *p.elite_idx);
        if (stop == kStopPending) {
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0)
                s_last = atomicAdd(p.ticket, 1u) == (unsigned int)a.inst_segs[sg.inst] - 1u ? 1 : 0;
            __syncthreads();
            if (s_last && threadIdx.x == 0) {
                *p.ticket = 0u;
                p.conv[2] = kStopped;
            }
        }
    }
}

// Stop states of a list of instances (the solve server reads them after each step).
__global__ void __launch_bounds__(kThreads) gather_stop_kernel(int32_t *const *conv, int32_t n,
                                                               int32_t *out)
{
    for (int32_t i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads)
        out[i] = conv[i][2];
}

// Generation 0 state: every qubit at theta = pi/4 (n = K), no elite, no best record.
__global__ void __launch_bounds__(kThreads) init_kernel(GenParams p, size_t state_words,
                                                        size_t xbytes, size_t acc_words)
{
    grid_dependency_wait();
    const uint32_t kk = (uint32_t)(4 * p.K) * (p.state8 ? 0x01010101u : 0x00010001u);
    uint32_t *s = reinterpret_cast<uint32_t *>(p.state);
    const size_t stride = (size_t)gridDim.x * kThreads;
    const size_t i0 = (size_t)blockIdx.x * kThreads + threadIdx.x;
    for (size_t i = i0; i < state_words; i += stride) s[i] = kk;
    for (size_t i = i0; i < xbytes; i += stride) p.xbits[i] = 0;
    for (size_t i = i0; i < (size_t)p.xstride; i += stride) p.best_row[i] = 0;
    for (size_t i = i0; i < acc_words; i += stride) p.acc[i] = 0ull;
    for (size_t i = i0; i < (size_t)p.np; i += stride) {
        p.fitness[i] = 0;
        p.cnt[i] = 0u;
    }
    if (p.fword) {   // no qubit at a bound: every fixed-vector word 0
        uint4 *f = reinterpret_cast<uint4 *>(p.fword);
        const size_t n = (size_t)p.np * (size_t)(p.fstride >> 5) / 4;
        for (size_t i = i0; i < n; i += stride) f[i] = make_uint4(0u, 0u, 0u, 0u);
        for (size_t i = i0; i < (size_t)p.np; i += stride) {
            p.fprev[i] = 0ull;
        }
        if (i0 == 0)
            for (int i = 0; i < 7; ++i) p.fcnt[i] = 0ull;
    }
    if (i0 == 0) {
        *p.gen = 0;
        *p.ticket = 0u;
        p.keys[0] = p.keys[1] = p.keys[2] = 0ull;
        p.qctr[0] = p.qctr[1] = p.qctr[2] = 0u;
        *p.elite_idx = 0;
        *p.bar_gen = 0;
        *p.error = 0;
        p.conv[0] = p.conv[1] = 0;
        p.conv[2] = kRunning;
        p.conv[3] = -1;
        p.best[0] = 0;
        p.best[1] = -1;
        p.best[2] = -1;
    }
}

__global__ void philox_kernel(const uint32_t *ck, uint32_t *out, int32_t n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t *q = ck + 6 * (size_t)i;
    const Draw4 r = philox4x32_10(q[0], q[1], q[2], q[3], q[4], q[5]);
    out[4 * (size_t)i + 0] = r.a;
    out[4 * (size_t)i + 1] = r.b;
    out[4 * (size_t)i + 2] = r.c;
    out[4 * (size_t)i + 3] = r.d;
}

}  // namespace qieo
