// qieo_noalloc.cu -- qieo_generation_noalloc: one QIEO generation on caller-owned device
// buffers, with the library's working memory in a fixed device array instead of an
// allocation.
//
// Some callers cannot call cudaMalloc at the point where they need a generation: code
// running while a memory pool is locked or being torn down, real-time loops where an
// allocation may stall, and hosts whose allocator owns every byte of device memory. They
// hold their own input and output buffers; this entry point needs nothing else from
// them. Its per-row sums and block counter live in g_noalloc_scratch below,
// a file-scope __device__ array of kNoallocScratchBytes that every GPU which loads the
// library keeps until the process exits.
//
// The host never dereferences g_noalloc_scratch: in host code that name is only a
// stand-in for the device symbol. The device address is looked up once per device with
// cudaGetSymbolAddress (with that device current) on the first call made on it, and is
// passed to the kernels. Device code reaches the array only through that pointer.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/qieo.h"
#include "qieo_device.cuh"

namespace qieo_internal {
void set_last_error(const char *msg);   // defined with qieo_last_error() in qieo_api.cu
}

namespace {

constexpr int kThreads = 256;
constexpr int kMaxD = 4000;
constexpr int kMaxThr = kMaxD / 2 + 1;

// Scratch layout: [0, 256) block counter; [256, 256 + 16 * kNoallocMaxNp) row sums
// (int64 weight sum, int64 value sum per chromosome).
constexpr size_t kCounterBytes = 256;
constexpr size_t kNoallocScratchBytes = kCounterBytes + 16 * (size_t)QIEO_NOALLOC_MAX_NP;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char *g_scratch_ptr[kMaxDevices];     // device address of g_noalloc_scratch

qieo_status noalloc_fail(qieo_status st, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
qieo_status noalloc_fail(qieo_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    qieo_internal::set_last_error(buf);   // read back through qieo_last_error()
    return st;
}

// Observation thresholds passed by value (kernel parameter space), so the call needs no
// copy into device memory either.
struct NoallocArgs {
    const int32_t *w, *v;
    int16_t *k;
    uint8_t *x;
    int64_t *fitness;
    int32_t *elite;
    unsigned int *counter;
    long long *sums;              // [2 np]
    int64_t capacity, lambda;
    int32_t ng, np, K, groups;    // groups = ceil(ng / 8) per row
    int32_t t, rule;
    uint32_t seed, inst;
    uint32_t thr[kMaxThr];        // low 32 bits of T[n]; T[2K] = 2^32 is handled as "always 1"
};

__global__ void __launch_bounds__(kThreads) noalloc_clear_kernel(unsigned int *counter,
                                                                 long long *sums, int32_t n)
{
    const int i = blockIdx.x * kThreads + threadIdx.x;
    if (i == 0) *counter = 0u;
    for (int j = i; j < n; j += gridDim.x * kThreads) sums[j] = 0;
}

// Observation and the per-chromosome sums of generation t on the caller's int16 angle
// indices, then (last block) the penalised fitness and the lowest-index elite.
__global__ void __launch_bounds__(kThreads) noalloc_observe_kernel(const NoallocArgs a)
{
    __shared__ uint32_t s_thr[kMaxThr];
    __shared__ int s_last;
    __shared__ int64_t s_f[kThreads / 32];
    __shared__ int32_t s_c[kThreads / 32];
    for (int i = threadIdx.x; i < 2 * a.K + 1; i += kThreads) s_thr[i] = a.thr[i];
    __syncthreads();

    const int64_t items = (int64_t)a.np * a.groups;
    for (int64_t it = (int64_t)blockIdx.x * kThreads + threadIdx.x; it < items;
         it += (int64_t)gridDim.x * kThreads) {
        const int32_t c = (int32_t)(it / a.groups);
        const int32_t g = (int32_t)(it - (int64_t)c * a.groups);
        const qieo::Draw4 d0 = qieo::philox4x32_10(2u * g, (uint32_t)c, (uint32_t)a.t, 0u, a.seed, a.inst);
        const qieo::Draw4 d1 = qieo::philox4x32_10(2u * g + 1u, (uint32_t)c, (uint32_t)a.t, 0u, a.seed, a.inst);
        const uint32_t u[8] = {d0.a, d0.b, d0.c, d0.d, d1.a, d1.b, d1.c, d1.d};
        long long sw = 0, sv = 0;
        for (int i = 0; i < 8; ++i) {
            const int32_t j = 8 * g + i;
            if (j >= a.ng) break;
            const size_t idx = (size_t)c * a.ng + j;
            // angle indices outside [-K, K] are invalid input; they are clamped so that
            // the table lookup stays inside the table
            const int32_t n = min(max((int32_t)a.k[idx] + a.K, 0), 2 * a.K);
            const bool x = n == 2 * a.K || u[i] < s_thr[n];
            a.x[idx] = x ? 1 : 0;
            if (x) {
                sw += a.w[j];
                sv += a.v[j];
            }
        }
        atomicAdd(reinterpret_cast<unsigned long long *>(a.sums + 2 * (size_t)c), (unsigned long long)sw);
        atomicAdd(reinterpret_cast<unsigned long long *>(a.sums + 2 * (size_t)c + 1), (unsigned long long)sv);
    }

    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(a.counter, 1u) == gridDim.x - 1u;
    __syncthreads();
    if (!s_last) return;
    __threadfence();

    int64_t bf = INT64_MIN;
    int32_t bc = 0x7fffffff;
    for (int c = threadIdx.x; c < a.np; c += kThreads) {
        const int64_t sw = __ldcg(a.sums + 2 * (size_t)c);
        const int64_t sv = __ldcg(a.sums + 2 * (size_t)c + 1);
        const int64_t f = sw <= a.capacity ? sv : -a.lambda * (sw - a.capacity);
        a.fitness[c] = f;
        if (f > bf) {
            bf = f;
            bc = c;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const int64_t of = __shfl_xor_sync(0xffffffffu, bf, o);
        const int32_t oc = __shfl_xor_sync(0xffffffffu, bc, o);
        if (of > bf || (of == bf && oc < bc)) {
            bf = of;
            bc = oc;
        }
    }
    if ((threadIdx.x & 31) == 0) {
        s_f[threadIdx.x >> 5] = bf;
        s_c[threadIdx.x >> 5] = bc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kThreads / 32; ++w)
            if (s_f[w] > bf || (s_f[w] == bf && s_c[w] < bc)) {
                bf = s_f[w];
                bc = s_c[w];
            }
        *a.elite = bc;
    }
}

// CIP of generation t: every angle index one step toward the elite's allele (rule R1), or
// only where the allele differs from the elite's (rule R2), saturating at -K and K.
__global__ void __launch_bounds__(kThreads) noalloc_cip_kernel(const NoallocArgs a)
{
    const int32_t e = *a.elite;
    const uint8_t *xe = a.x + (size_t)e * a.ng;
    const size_t total = (size_t)a.np * a.ng;
    for (size_t idx = (size_t)blockIdx.x * kThreads + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * kThreads) {
        const size_t j = idx % (size_t)a.ng;
        const int xe_j = xe[j];
        if (a.rule == 1 && a.x[idx] == xe_j) continue;
        const int32_t kn = (int32_t)a.k[idx] + (xe_j ? 1 : -1);
        if (kn >= -a.K && kn <= a.K) a.k[idx] = (int16_t)kn;
    }
}

// Device address of g_noalloc_scratch on the current device (looked up once per device).
qieo_status scratch_address(unsigned char **out, int *device)
{
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return noalloc_fail(QIEO_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(ce));
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(QIEO_ERR_INVALID, "device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        ce = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (ce != cudaSuccess || !p)
            return noalloc_fail(QIEO_ERR_CUDA, "cudaGetSymbolAddress(g_noalloc_scratch): %s",
                                cudaGetErrorString(ce));
        g_scratch_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_ptr[dev];
    *device = dev;
    return QIEO_OK;
}

}  // namespace

extern "C" qieo_status qieo_generation_noalloc(const qieo_problem *problem, const qieo_params *params,
                                               int32_t t, int16_t *k, uint8_t *x, int64_t *fitness,
                                               int32_t *elite)
{
    if (!problem || !params || !k || !x || !fitness || !elite || !problem->weights || !problem->values)
        return noalloc_fail(QIEO_ERR_INVALID, "NULL argument");
    const int32_t ng = problem->ng, np = params->np, D = params->dtheta_den;
    if (ng < 1) return noalloc_fail(QIEO_ERR_INVALID, "ng must be >= 1 (got %d)", ng);
    if (np < 1 || np > QIEO_NOALLOC_MAX_NP)
        return noalloc_fail(QIEO_ERR_INVALID,
                            "np must be in [1, %d] (the size of the static scratch array); got %d",
                            QIEO_NOALLOC_MAX_NP, np);
    if (D < 4 || D > kMaxD || D % 4 != 0)
        return noalloc_fail(QIEO_ERR_INVALID, "dtheta_den must be a multiple of 4 in [4, %d]", kMaxD);
    if (params->penalty_lambda < 1) return noalloc_fail(QIEO_ERR_INVALID, "penalty_lambda must be >= 1");
    if (params->rotate_rule != QIEO_RULE_R1 && params->rotate_rule != QIEO_RULE_R2)
        return noalloc_fail(QIEO_ERR_INVALID, "rotate_rule must be 0 or 1");
    if (problem->capacity < 0) return noalloc_fail(QIEO_ERR_INVALID, "capacity must be >= 0");
    if (t < 0) return noalloc_fail(QIEO_ERR_INVALID, "generation t must be >= 0");
    if ((int64_t)np * ng > ((int64_t)1 << 40)) return noalloc_fail(QIEO_ERR_INVALID, "np * ng too large");

    unsigned char *scratch = nullptr;
    int dev = 0;
    qieo_status st = scratch_address(&scratch, &dev);
    if (st != QIEO_OK) return st;

    NoallocArgs a;
    std::memset(&a, 0, sizeof a);
    a.w = problem->weights;
    a.v = problem->values;
    a.k = k;
    a.x = x;
    a.fitness = fitness;
    a.elite = elite;
    a.counter = reinterpret_cast<unsigned int *>(scratch);
    a.sums = reinterpret_cast<long long *>(scratch + kCounterBytes);
    a.capacity = problem->capacity;
    a.lambda = params->penalty_lambda;
    a.ng = ng;
    a.np = np;
    a.K = D / 4;
    a.groups = (ng + 7) / 8;
    a.t = t;
    a.rule = params->rotate_rule;
    a.seed = params->seed;
    a.inst = params->instance_id;
    // T[n] = round(sin^2(n pi / D) 2^32) = round(2^31 (1 - cos(2 pi n / D))) for n <= K,
    // mirrored above (T[2K - n] = 2^32 - T[n]); T[0] = 0 and T[K] = 2^31 exactly.
    const long double pi = acosl(-1.0L);
    for (int32_t n = 0; n <= a.K; ++n) {
        const long double val = 2147483648.0L * (1.0L - cosl(2.0L * pi * n / D));
        a.thr[n] = (uint32_t)llroundl(val);
    }
    a.thr[0] = 0u;
    a.thr[a.K] = 1u << 31;
    for (int32_t n = a.K + 1; n <= 2 * a.K; ++n)
        a.thr[n] = (uint32_t)((1ull << 32) - a.thr[2 * a.K - n]);

    int sms = 0;
    cudaError_t ce = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (ce != cudaSuccess) return noalloc_fail(QIEO_ERR_CUDA, "device query: %s", cudaGetErrorString(ce));
    cudaStream_t s = static_cast<cudaStream_t>(params->stream);
    const int clear_blocks = (int)std::min<int64_t>(((int64_t)2 * np + kThreads - 1) / kThreads, 1024);
    noalloc_clear_kernel<<<clear_blocks, kThreads, 0, s>>>(a.counter, a.sums, 2 * np);
    const int64_t items = (int64_t)np * a.groups;
    const int obs_blocks = (int)std::max<int64_t>(1, std::min<int64_t>((items + kThreads - 1) / kThreads, 4 * (int64_t)sms));
    noalloc_observe_kernel<<<obs_blocks, kThreads, 0, s>>>(a);
    const int64_t total = (int64_t)np * ng;
    const int cip_blocks = (int)std::max<int64_t>(1, std::min<int64_t>((total + kThreads - 1) / kThreads, 8 * (int64_t)sms));
    noalloc_cip_kernel<<<cip_blocks, kThreads, 0, s>>>(a);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) return noalloc_fail(QIEO_ERR_CUDA, "launch: %s", cudaGetErrorString(ce));
    return QIEO_OK;
}
