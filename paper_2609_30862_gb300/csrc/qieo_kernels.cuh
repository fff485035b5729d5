// qieo_kernels.cuh -- device code of the GB300 QIEO library.
//
// One fused kernel per generation (Sec. III-B, Fig. 1 of arxiv 2609.30862):
//   CIP(t-1)  rotate every qubit one step toward the previous elite's allele,
//   QIP(t)    observe every qubit against a Philox draw,
//   FE(t)     eq. (1) weight/value sums per chromosome (segmented reduction over genes),
//   DE(t)     the last thread block to finish picks the generation-best chromosome.
// The CIP of generation t is applied at the top of generation t+1 because the elite is a
// grid-wide result; qieo_run applies the CIP of its last generation with cip_kernel.
//
// Data layout in device memory (row c = chromosome c, gene-fastest, Sec. V-D):
//   state  uint16 n = k + K in [0, 2K], rows padded to a multiple of 8 genes; one uint4
//          ("vector") holds 8 genes, and a uint32 lane of it holds 2 genes (pair).
//   xbits  one byte per vector: bit i = allele of gene 8v + i; rows padded to 16 bytes.
//   items  narrow: uint32 (v << 16 | w) per gene; wide: int32 w[], int32 v[].
//   acc    narrow: uint64 (SV << 32 | SW) per row; wide: int64 SW, SV per row.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace qieo {

constexpr int kThreads = 256;

// ---------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC 2011). One round maps (c0, c1, c2, c3)
// to (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)); the key advances by
// the Weyl increments between rounds. The 32x32->64 products map to one wide multiply.
// ---------------------------------------------------------------------------------------
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

struct Draw4 {
    uint32_t a, b, c, d;
};

__device__ __forceinline__ Draw4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                               uint32_t c3, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)kPhiloxM0 * (uint64_t)c0;
        const uint64_t p1 = (uint64_t)kPhiloxM1 * (uint64_t)c2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        c1 = (uint32_t)p1;
        c3 = (uint32_t)p0;
        c0 = n0;
        c2 = n2;
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    return {c0, c1, c2, c3};
}

// ---------------------------------------------------------------------------------------
// CIP on a pair of biased angle indices held in one uint32 (gene 2i low, 2i+1 high).
// d per half: 2 = step toward allele 1, 0 = step toward allele 0, 1 = no move.
// n' = min(max(n + d, 1) - 1, 2K): saturates theta at 0 and pi/2 (the bounds of the
// angle index). No half can carry into the other: n + d <= 2K + 2 < 2^16.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t delta_pair(uint32_t e2, uint32_t m2)
{
    // e2: elite alleles of the two genes (bit 0, bit 1); m2: which of them move.
    const uint32_t lo = 1u - (m2 & 1u) + ((m2 & e2 & 1u) << 1);
    const uint32_t hi = 1u - ((m2 >> 1) & 1u) + ((((m2 & e2) >> 1) & 1u) << 1);
    return lo | (hi << 16);
}

__device__ __forceinline__ uint32_t rotate_pair(uint32_t s, uint32_t d, uint32_t kk2)
{
    return __vminu2(__vmaxu2(s + d, 0x00010001u) - 0x00010001u, kk2);
}

__device__ __forceinline__ uint4 rotate_vec(uint4 s, uint32_t e8, uint32_t m8, uint32_t kk2)
{
    s.x = rotate_pair(s.x, delta_pair(e8 & 3u, m8 & 3u), kk2);
    s.y = rotate_pair(s.y, delta_pair((e8 >> 2) & 3u, (m8 >> 2) & 3u), kk2);
    s.z = rotate_pair(s.z, delta_pair((e8 >> 4) & 3u, (m8 >> 4) & 3u), kk2);
    s.w = rotate_pair(s.w, delta_pair((e8 >> 6) & 3u, (m8 >> 6) & 3u), kk2);
    return s;
}

struct GenParams {
    uint4 *state;                 // [np][svec]
    uint8_t *xbits;               // [np][xstride]
    const uint4 *items_narrow;    // [2 svec] packed (v << 16 | w), 4 genes per uint4
    const int4 *w4;               // wide: [2 svec] weights
    const int4 *v4;               // wide: [2 svec] values
    uint8_t *elite;               // [xstride] alleles of the last elite
    unsigned long long *acc;      // narrow [np]; wide [2 np]
    int64_t *fitness;             // [np] of the last generation
    int32_t *hist_e;              // [capacity] elite index per generation
    int64_t *hist_f;              // [capacity] elite fitness per generation
    int64_t *best;                // [3] fitness, generation (-1 none), chromosome
    uint8_t *best_row;            // [xstride]
    int32_t *gen;                 // number of the generation to run next
    unsigned int *ticket;         // blocks finished in this generation
    const uint32_t *thr;          // [2K+1] low 32 bits of T[n] (T[2K] = 2^32 -> 0)
    int32_t np, svec, xstride, K;
    int64_t capacity, lambda;
    uint32_t key0, key1;
    int32_t lanes, warps, rows_per_cta;
    int32_t apply_cip, do_de;
};

// Row-wise DetermineElite, run by the last block of a generation: eq. (1) from the row
// sums, lowest-index argmax, elite/best records, and the accumulators cleared for the next
// generation.
template <bool kNarrow>
__device__ void determine_elite(const GenParams &p, int32_t t)
{
    __shared__ int64_t s_f[kThreads / 32];
    __shared__ int32_t s_c[kThreads / 32];
    __shared__ int32_t s_e;
    __shared__ int32_t s_improved;
    const int tid = threadIdx.x;

    int64_t bf = INT64_MIN;
    int32_t bc = 0x7fffffff;
    for (int c = tid; c < p.np; c += kThreads) {
        int64_t sw, sv;
        if (kNarrow) {
            const unsigned long long a = __ldcg(p.acc + c);
            sw = (int64_t)(a & 0xffffffffull);
            sv = (int64_t)(a >> 32);
            p.acc[c] = 0ull;
        } else {
            sw = (int64_t)__ldcg(p.acc + 2 * (size_t)c);
            sv = (int64_t)__ldcg(p.acc + 2 * (size_t)c + 1);
            p.acc[2 * (size_t)c] = 0ull;
            p.acc[2 * (size_t)c + 1] = 0ull;
        }
        const int64_t f = sw <= p.capacity ? sv : -p.lambda * (sw - p.capacity);
        p.fitness[c] = f;
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
        p.hist_e[t] = bc;
        p.hist_f[t] = bf;
        const int improved = (p.best[1] < 0 || bf > p.best[0]) ? 1 : 0;
        if (improved) {
            p.best[0] = bf;
            p.best[1] = t;
            p.best[2] = bc;
        }
        s_e = bc;
        s_improved = improved;
    }
    __syncthreads();
    const int32_t e = s_e;
    const int improved = s_improved;
    const uint4 *src = reinterpret_cast<const uint4 *>(p.xbits + (size_t)e * p.xstride);
    uint4 *dst = reinterpret_cast<uint4 *>(p.elite);
    uint4 *bdst = reinterpret_cast<uint4 *>(p.best_row);
    for (int i = tid; i < p.xstride / 16; i += kThreads) {
        const uint4 v = __ldcg(src + i);
        dst[i] = v;
        if (improved) bdst[i] = v;
    }
    if (tid == 0) {
        *p.gen = t + 1;
        *p.ticket = 0u;
    }
}

// ---------------------------------------------------------------------------------------
// The fused generation kernel. Grid: x = gene tiles of lanes*warps vectors, y = chunks of
// rows_per_cta chromosomes. Thread (r_sub, v_in) of a block handles vector v_in of rows
// r_sub, r_sub + rows_per_pass, ... of its chunk; its 8 items stay in registers for all
// of them. Row sums are reduced over the lanes of a segment by shuffles, over the warps of
// a tile in shared memory, and over tiles by one 64-bit atomic per row and block.
// ---------------------------------------------------------------------------------------
template <bool kNarrow, int kRule>
__global__ void __launch_bounds__(kThreads, 2) generation_kernel(const GenParams p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_last;
    const int n_thr = 2 * p.K + 1;
    uint32_t *s_thr = reinterpret_cast<uint32_t *>(smem_raw);
    unsigned long long *s_acc64 =
        reinterpret_cast<unsigned long long *>(smem_raw + (((size_t)n_thr * 4 + 15) & ~(size_t)15));
    uint32_t *s_acc32 = reinterpret_cast<uint32_t *>(s_acc64);

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int tile_vecs = p.lanes * p.warps;
    const int rows_per_pass = kThreads / tile_vecs;
    const int r_sub = tid / tile_vecs;
    const int v_in = tid - r_sub * tile_vecs;
    const int vec = blockIdx.x * tile_vecs + v_in;
    const bool active = vec < p.svec;
    const int row0 = blockIdx.y * p.rows_per_cta;
    const int rows_here = min(p.rows_per_cta, p.np - row0);
    const int passes = (rows_here + rows_per_pass - 1) / rows_per_pass;

    for (int i = tid; i < n_thr; i += kThreads) s_thr[i] = p.thr[i];
    for (int i = tid; i < 2 * rows_here; i += kThreads) {
        if (kNarrow) s_acc32[i] = 0u;
        else s_acc64[i] = 0ull;
    }
    const int32_t t = *p.gen;

    // Items of this thread's 8 genes (zero outside the row: they add nothing).
    uint32_t wv[8];
    int32_t wi[8], vi[8];
    if (kNarrow) {
        uint4 a = make_uint4(0, 0, 0, 0), b = a;
        if (active) {
            a = __ldg(p.items_narrow + 2 * (size_t)vec);
            b = __ldg(p.items_narrow + 2 * (size_t)vec + 1);
        }
        wv[0] = a.x; wv[1] = a.y; wv[2] = a.z; wv[3] = a.w;
        wv[4] = b.x; wv[5] = b.y; wv[6] = b.z; wv[7] = b.w;
    } else {
        int4 a = make_int4(0, 0, 0, 0), b = a, c = a, d = a;
        if (active) {
            a = __ldg(p.w4 + 2 * (size_t)vec);
            b = __ldg(p.w4 + 2 * (size_t)vec + 1);
            c = __ldg(p.v4 + 2 * (size_t)vec);
            d = __ldg(p.v4 + 2 * (size_t)vec + 1);
        }
        wi[0] = a.x; wi[1] = a.y; wi[2] = a.z; wi[3] = a.w;
        wi[4] = b.x; wi[5] = b.y; wi[6] = b.z; wi[7] = b.w;
        vi[0] = c.x; vi[1] = c.y; vi[2] = c.z; vi[3] = c.w;
        vi[4] = d.x; vi[5] = d.y; vi[6] = d.z; vi[7] = d.w;
    }
    const uint32_t e8 = (p.apply_cip && active) ? (uint32_t)p.elite[vec] : 0u;
    const uint32_t kk2 = (uint32_t)(2 * p.K) * 0x00010001u;
    const uint32_t n_top = (uint32_t)(2 * p.K);
    __syncthreads();

    for (int pass = 0; pass < passes; ++pass) {
        const int rr = pass * rows_per_pass + r_sub;
        const bool row_ok = rr < rows_here;
        const bool live = active && row_ok;
        const int c = row0 + rr;
        const size_t sidx = (size_t)c * p.svec + vec;
        const size_t xidx = (size_t)c * p.xstride + vec;

        uint4 s = make_uint4(0, 0, 0, 0);
        if (live) s = p.state[sidx];
        if (p.apply_cip) {
            uint32_t m8 = 0xffu;                               // R1: every qubit moves
            if (kRule == 1) m8 = live ? (e8 ^ (uint32_t)p.xbits[xidx]) : 0u;
            s = rotate_vec(s, e8, m8, kk2);
        }

        const uint32_t ctr0 = 2u * (uint32_t)vec;
        const Draw4 r0 = philox4x32_10(ctr0, (uint32_t)c, (uint32_t)t, 0u, p.key0, p.key1);
        const Draw4 r1 = philox4x32_10(ctr0 + 1u, (uint32_t)c, (uint32_t)t, 0u, p.key0, p.key1);
        const uint32_t u[8] = {r0.a, r0.b, r0.c, r0.d, r1.a, r1.b, r1.c, r1.d};
        const uint32_t sp[4] = {s.x, s.y, s.z, s.w};

        uint32_t xb = 0u;
        uint32_t accn = 0u;
        int64_t acw = 0, acv = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const uint32_t n = (i & 1) ? (sp[i >> 1] >> 16) : (sp[i >> 1] & 0xffffu);
            const bool x = (u[i] < s_thr[n]) || (n == n_top);
            if (x) {
                xb |= 1u << i;
                if (kNarrow) {
                    accn += wv[i];
                } else {
                    acw += wi[i];
                    acv += vi[i];
                }
            }
        }
        if (live) {
            p.state[sidx] = s;
            p.xbits[xidx] = (uint8_t)xb;
        }

        // Segment (row) reduction over p.lanes lanes.
        for (int o = p.lanes >> 1; o > 0; o >>= 1) {
            if (kNarrow) {
                accn += __shfl_xor_sync(0xffffffffu, accn, o);
            } else {
                acw += __shfl_xor_sync(0xffffffffu, acw, o);
                acv += __shfl_xor_sync(0xffffffffu, acv, o);
            }
        }
        if (row_ok && (lane & (p.lanes - 1)) == 0) {
            if (kNarrow) {
                atomicAdd(s_acc32 + 2 * rr, accn & 0xffffu);
                atomicAdd(s_acc32 + 2 * rr + 1, accn >> 16);
            } else {
                atomicAdd(s_acc64 + 2 * rr, (unsigned long long)acw);
                atomicAdd(s_acc64 + 2 * rr + 1, (unsigned long long)acv);
            }
        }
    }
    __syncthreads();
    for (int i = tid; i < rows_here; i += kThreads) {
        if (kNarrow) {
            const unsigned long long v =
                ((unsigned long long)s_acc32[2 * i + 1] << 32) | (unsigned long long)s_acc32[2 * i];
            atomicAdd(p.acc + row0 + i, v);
        } else {
            atomicAdd(p.acc + 2 * (size_t)(row0 + i), s_acc64[2 * i]);
            atomicAdd(p.acc + 2 * (size_t)(row0 + i) + 1, s_acc64[2 * i + 1]);
        }
    }
    if (!p.do_de) return;

    // Last block to finish runs DetermineElite (no block waits for another).
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        const unsigned int prev = atomicAdd(p.ticket, 1u);
        s_last = (prev == gridDim.x * gridDim.y - 1u) ? 1 : 0;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    determine_elite<kNarrow>(p, t);
}

// DetermineElite for the host variant: the elite index e comes from the host; this kernel
// writes the records exactly as the fused path does (one block).
template <bool kNarrow>
__global__ void __launch_bounds__(kThreads) record_elite_kernel(const GenParams p, int32_t e)
{
    __shared__ int s_improved;
    const int tid = threadIdx.x;
    const int32_t t = *p.gen;
    for (int c = tid; c < p.np; c += kThreads) {
        int64_t sw, sv;
        if (kNarrow) {
            const unsigned long long a = p.acc[c];
            sw = (int64_t)(a & 0xffffffffull);
            sv = (int64_t)(a >> 32);
            p.acc[c] = 0ull;
        } else {
            sw = (int64_t)p.acc[2 * (size_t)c];
            sv = (int64_t)p.acc[2 * (size_t)c + 1];
            p.acc[2 * (size_t)c] = 0ull;
            p.acc[2 * (size_t)c + 1] = 0ull;
        }
        p.fitness[c] = sw <= p.capacity ? sv : -p.lambda * (sw - p.capacity);
    }
    __syncthreads();
    if (tid == 0) {
        const int64_t fe = p.fitness[e];
        p.hist_e[t] = e;
        p.hist_f[t] = fe;
        const int improved = (p.best[1] < 0 || fe > p.best[0]) ? 1 : 0;
        if (improved) {
            p.best[0] = fe;
            p.best[1] = t;
            p.best[2] = e;
        }
        s_improved = improved;
    }
    __syncthreads();
    const uint4 *src = reinterpret_cast<const uint4 *>(p.xbits + (size_t)e * p.xstride);
    for (int i = tid; i < p.xstride / 16; i += kThreads) {
        const uint4 v = src[i];
        reinterpret_cast<uint4 *>(p.elite)[i] = v;
        if (s_improved) reinterpret_cast<uint4 *>(p.best_row)[i] = v;
    }
    if (tid == 0) *p.gen = t + 1;
}

// CIP of the last generation of a run (the same rotation the next generation would fuse).
template <int kRule>
__global__ void __launch_bounds__(kThreads) cip_kernel(uint4 *state, const uint8_t *xbits,
                                                       const uint8_t *elite, int32_t np,
                                                       int32_t svec, int32_t xstride, int32_t K)
{
    const uint32_t kk2 = (uint32_t)(2 * K) * 0x00010001u;
    const size_t total = (size_t)np * svec;
    for (size_t i = (size_t)blockIdx.x * kThreads + threadIdx.x; i < total;
         i += (size_t)gridDim.x * kThreads) {
        const size_t c = i / (size_t)svec;
        const size_t v = i - c * (size_t)svec;
        const uint32_t e8 = elite[v];
        const uint32_t m8 = kRule == 1 ? (e8 ^ (uint32_t)xbits[c * xstride + v]) : 0xffu;
        state[i] = rotate_vec(state[i], e8, m8, kk2);
    }
}

// Generation 0 state: every qubit at theta = pi/4 (n = K), no elite, no best record.
__global__ void __launch_bounds__(kThreads) init_kernel(GenParams p, size_t state_words,
                                                        size_t xbytes)
{
    const uint32_t kk = (uint32_t)p.K * 0x00010001u;
    uint32_t *s = reinterpret_cast<uint32_t *>(p.state);
    const size_t stride = (size_t)gridDim.x * kThreads;
    const size_t i0 = (size_t)blockIdx.x * kThreads + threadIdx.x;
    for (size_t i = i0; i < state_words; i += stride) s[i] = kk;
    for (size_t i = i0; i < xbytes; i += stride) p.xbits[i] = 0;
    for (size_t i = i0; i < (size_t)p.xstride; i += stride) {
        p.elite[i] = 0;
        p.best_row[i] = 0;
    }
    const size_t nacc = (size_t)p.np * 2;
    for (size_t i = i0; i < nacc; i += stride) p.acc[i] = 0ull;
    for (size_t i = i0; i < (size_t)p.np; i += stride) p.fitness[i] = 0;
    if (i0 == 0) {
        *p.gen = 0;
        *p.ticket = 0u;
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
