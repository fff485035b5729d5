// qieo_ceiling.cu -- measured integer ceiling of the generation kernel's per-gene work.
//
// The fused generation kernel moves 4 bytes of state per gene-update (the int16 angle index
// read and written) and does, per gene-update, a quarter of a Philox4x32-10 call, the CIP
// rotation, the threshold compare, the allele bit and the packed item add. Which of the two
// bounds it is set by the integer pipes, not by a nominal lane count: the 32x32->64
// multiplies of Philox run on a half-rate pipe at a fraction of the simple-integer rate, and
// the compiler's instruction mix decides how the rest share the issue slots. This file
// measures that ceiling on the device itself: the same per-gene arithmetic the drawn pass
// of the generation kernel does (the same helpers: rotate_pair_signed, philox4x32_10_rk
// with the round keys in the parameter block, the shared-memory threshold table), with the
// state held in registers instead of streamed from memory, no per-row reduction and no
// stores but one word per thread at the end. A second kernel runs Philox4x32-10 alone.
//
// Both kernels use the generation kernel's launch shape (256 threads, three blocks per SM,
// one block per SM-slot) and draw with the same counters (gene vector, chromosome,
// generation), so the compiler can hoist the same loop-invariant rounds it hoists there.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <vector>

#include "../../include/qieo.h"
#include "qieo_device.cuh"

namespace qieo_internal {
void set_last_error(const char *msg);                           // qieo_api.cu
void build_thresholds(int32_t D, std::vector<uint64_t> &T);   // qieo_api.cu
}

namespace {

constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 3;
constexpr int kD = 100;               // the named workloads' rotation step pi/100
constexpr int kK = kD / 4;

struct CeilingParams {
    uint32_t *sink;                   // [grid * kThreads] one word per thread
    const uint32_t *thr;              // [2K + 1] low 32 bits of T[n]
    int32_t passes;                   // 8-gene passes per thread
    int32_t t;                        // generation number of the draws
    uint32_t rk0[10], rk1[10];        // Philox round keys
};

qieo_status ceil_fail(qieo_status st, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
qieo_status ceil_fail(qieo_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    qieo_internal::set_last_error(buf);
    return st;
}

#define CEIL_TRY(expr)                                                                        \
    do {                                                                                      \
        cudaError_t err_ = (expr);                                                            \
        if (err_ != cudaSuccess)                                                              \
            return ceil_fail(err_ == cudaErrorMemoryAllocation ? QIEO_ERR_OOM : QIEO_ERR_CUDA, \
                             "%s: %s", #expr, cudaGetErrorString(err_));                      \
    } while (0)

// The drawn pass's per-gene arithmetic over `passes` rows of one 8-gene vector per thread:
// CIP toward a fixed elite pattern (rule R1 signed steps formed once, as the generation
// kernel forms them once per segment), two Philox4x32-10 calls keyed (2 vec + i, row, t),
// eight table lookups and compares, the allele byte and the packed (v << 16 | w) item sums.
__global__ void __launch_bounds__(kThreads, kBlocksPerSm) drawn_ceiling_kernel(const CeilingParams p)
{
    __shared__ uint32_t s_thr[2 * kK + 1];
    for (int i = threadIdx.x; i < 2 * kK + 1; i += kThreads) s_thr[i] = p.thr[i];
    __syncthreads();
    const unsigned char *thr_bytes = reinterpret_cast<const unsigned char *>(s_thr);
    const uint32_t vec = blockIdx.x * kThreads + threadIdx.x;
    uint32_t wv[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const uint32_t w = 1u + (vec * 8u + (uint32_t)i) % 10u;
        wv[i] = ((w + 5u) << 16) | w;
    }
    const uint32_t e8 = (vec * 37u + 11u) & 0xffu;
    const uint32_t d0 = qieo::signed_step(qieo::delta_pair(e8 & 3u, 3u));
    const uint32_t d1 = qieo::signed_step(qieo::delta_pair((e8 >> 2) & 3u, 3u));
    const uint32_t d2 = qieo::signed_step(qieo::delta_pair((e8 >> 4) & 3u, 3u));
    const uint32_t d3 = qieo::signed_step(qieo::delta_pair((e8 >> 6) & 3u, 3u));
    const uint32_t off_top = 8u * kK;
    const uint32_t k8 = off_top * 0x00010001u;
    uint4 s = make_uint4(4u * kK * 0x00010001u, 4u * kK * 0x00010001u, 4u * kK * 0x00010001u,
                         4u * kK * 0x00010001u);
    const uint32_t ctr0 = 2u * vec;
    const uint32_t row0 = blockIdx.x * 7u;
    uint32_t chk = 0u;
    for (int pass = 0; pass < p.passes; ++pass) {
        s.x = qieo::rotate_pair_signed(s.x, d0, k8);
        s.y = qieo::rotate_pair_signed(s.y, d1, k8);
        s.z = qieo::rotate_pair_signed(s.z, d2, k8);
        s.w = qieo::rotate_pair_signed(s.w, d3, k8);
        const uint32_t c = row0 + (uint32_t)pass;
        const qieo::Draw4 r0 = qieo::philox4x32_10_rk(ctr0, c, (uint32_t)p.t, 0u, p.rk0, p.rk1);
        const qieo::Draw4 r1 = qieo::philox4x32_10_rk(ctr0 + 1u, c, (uint32_t)p.t, 0u, p.rk0, p.rk1);
        const uint32_t u[8] = {r0.a, r0.b, r0.c, r0.d, r1.a, r1.b, r1.c, r1.d};
        const uint32_t sp[4] = {s.x, s.y, s.z, s.w};
        uint32_t xbits = 0u, accn = 0u;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const uint32_t off = (i & 1) ? (sp[i >> 1] >> 16) : (sp[i >> 1] & 0xffffu);
            const uint32_t thr = *reinterpret_cast<const uint32_t *>(thr_bytes + off);
            if ((u[i] < thr) || (off == off_top)) {
                xbits |= 1u << i;
                accn += wv[i];
            }
        }
        chk += accn ^ (xbits << 24);
    }
    p.sink[vec] = chk ^ s.x ^ s.y ^ s.z ^ s.w;
}

// Philox4x32-10 alone: two calls per 8-gene pass with the same counters, the eight words
// folded into one (three-input xors).
__global__ void __launch_bounds__(kThreads, kBlocksPerSm) philox_ceiling_kernel(const CeilingParams p)
{
    const uint32_t vec = blockIdx.x * kThreads + threadIdx.x;
    const uint32_t ctr0 = 2u * vec;
    const uint32_t row0 = blockIdx.x * 7u;
    uint32_t chk = 0u;
    for (int pass = 0; pass < p.passes; ++pass) {
        const uint32_t c = row0 + (uint32_t)pass;
        const qieo::Draw4 r0 = qieo::philox4x32_10_rk(ctr0, c, (uint32_t)p.t, 0u, p.rk0, p.rk1);
        const qieo::Draw4 r1 = qieo::philox4x32_10_rk(ctr0 + 1u, c, (uint32_t)p.t, 0u, p.rk0, p.rk1);
        chk ^= r0.a ^ r0.b ^ r0.c ^ r0.d ^ r1.a ^ r1.b ^ r1.c ^ r1.d;
    }
    p.sink[vec] = chk;
}

}  // namespace

extern "C" {

qieo_status qieo_measure_integer_ceiling(int32_t reps, qieo_integer_ceiling *out)
{
    if (!out) return ceil_fail(QIEO_ERR_INVALID, "out is NULL");
    if (reps < 1 || reps > 1000) return ceil_fail(QIEO_ERR_INVALID, "reps must be in [1, 1000] (got %d)", reps);
    int dev = 0, sms = 0;
    CEIL_TRY(cudaGetDevice(&dev));
    CEIL_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = std::max(1, sms) * kBlocksPerSm;
    const int32_t passes = 2048;

    std::vector<uint64_t> T;
    qieo_internal::build_thresholds(kD, T);
    std::vector<uint32_t> thr(T.size());
    for (size_t i = 0; i < T.size(); ++i) thr[i] = (uint32_t)T[i];   // T[2K] = 2^32 -> 0

    CeilingParams p{};
    p.passes = passes;
    p.t = 7;
    uint32_t k0 = 1u, k1 = 0u;                        // seed 1, instance 0
    for (int r = 0; r < 10; ++r) {
        p.rk0[r] = k0;
        p.rk1[r] = k1;
        k0 += qieo::kPhiloxW0;
        k1 += qieo::kPhiloxW1;
    }

    cudaStream_t stream = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    void *mem = nullptr;
    qieo_status st = QIEO_OK;
    auto fin = [&](qieo_status s) {
        if (stream) cudaStreamSynchronize(stream);
        if (mem) cudaFree(mem);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (stream) cudaStreamDestroy(stream);
        return s;
    };
    cudaError_t ce = cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    if (ce == cudaSuccess) ce = cudaMalloc(&mem, (size_t)grid * kThreads * sizeof(uint32_t) + 4096);
    if (ce != cudaSuccess)
        return fin(ceil_fail(ce == cudaErrorMemoryAllocation ? QIEO_ERR_OOM : QIEO_ERR_CUDA, "setup: %s",
                             cudaGetErrorString(ce)));
    p.thr = reinterpret_cast<const uint32_t *>(mem);
    p.sink = reinterpret_cast<uint32_t *>(static_cast<unsigned char *>(mem) + 4096);
    ce = cudaMemcpyAsync(mem, thr.data(), thr.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, stream);
    if (ce != cudaSuccess) return fin(ceil_fail(QIEO_ERR_CUDA, "table upload: %s", cudaGetErrorString(ce)));

    const double genes = (double)grid * kThreads * passes * 8.0;
    double best[2] = {0.0, 0.0};
    for (int kind = 0; kind < 2 && st == QIEO_OK; ++kind) {
        for (int r = 0; r <= reps; ++r) {          // the first launch warms up
            cudaEventRecord(e0, stream);
            if (kind == 0) drawn_ceiling_kernel<<<grid, kThreads, 0, stream>>>(p);
            else philox_ceiling_kernel<<<grid, kThreads, 0, stream>>>(p);
            cudaEventRecord(e1, stream);
            ce = cudaEventSynchronize(e1);
            if (ce == cudaSuccess) ce = cudaGetLastError();
            if (ce != cudaSuccess) {
                st = ceil_fail(QIEO_ERR_CUDA, "ceiling kernel: %s", cudaGetErrorString(ce));
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (r > 0 && ms > 0.f) best[kind] = std::max(best[kind], genes / (ms * 1e-3));
        }
    }
    if (st != QIEO_OK) return fin(st);
    out->drawn_genes_per_s = best[0];
    out->philox_genes_per_s = best[1];
    out->genes_per_launch = (int64_t)genes;
    out->grid_ctas = grid;
    out->reps = reps;
    return fin(QIEO_OK);
}

}  // extern "C"
