// lskum_q_derivatives_noalloc: q-derivatives with every scratch buffer in one
// statically sized __device__ array, so the call allocates no device memory.
// It serves callers that cannot allocate where they call from (a caching
// allocator that owns the GPU's memory, a loop that must not pay the device
// synchronisation of cudaMalloc/cudaFree, a fixed memory budget). The paper
// has no counterpart; this is a plumbing variant of lskum_q_derivatives.
//
// Arithmetic: the q-variables from U, then the least-squares q-derivatives
// (the first-order solve, then Jacobi inner iterations on the corrected
// differences) in the global frame, the 2x2 sums formed on the fly from the
// coordinates (no precomputed weights).
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "lskum.h"
#include "lskum_device.cuh"
#include "lskum_kernels.h"

namespace lskum {

// scratch layout (doubles): [0, 32) status words, then q [n][4], ga [n][8],
// gb [n][8] for up to LSKUM_NOALLOC_MAX_POINTS points
static constexpr int64_t kNoallocHeader = 32;
static constexpr int64_t kNoallocPerPoint = 4 + 8 + 8;
static __device__ __align__(256) double g_noalloc_scratch[kNoallocHeader + kNoallocPerPoint * LSKUM_NOALLOC_MAX_POINTS];

// status word bits (int view of the header)
enum : int { NA_NONPHYSICAL = 1, NA_BAD_INDEX = 2, NA_BAD_OFFSETS = 4 };

__global__ void __launch_bounds__(256) k_na_q(int64_t n, Gas gas, const double *__restrict__ U,
                                              double *__restrict__ q, int *status)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    double u[4] = {U[p], U[n + p], U[2 * n + p], U[3 * n + p]}, qq[4];
    if (!q_from_U(u, gas, qq)) atomicOr(status, NA_NONPHYSICAL);
    store4(q, p, qq);
}

// One least-squares solve at every point. g_old == nullptr: first order. Output to
// g_new ([n][8] scratch) or, on the final pass, to qx/qy ([4][n], caller).
__global__ void __launch_bounds__(128) k_na_grad(int64_t n, const double *__restrict__ x,
                                                 const double *__restrict__ y,
                                                 const int32_t *__restrict__ off,
                                                 const int32_t *__restrict__ idx,
                                                 const double *__restrict__ q,
                                                 const double *__restrict__ g_old,
                                                 double *__restrict__ g_new, double *__restrict__ qx,
                                                 double *__restrict__ qy, int *status)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    double q0[4], g0[8];
    load4(q, p, q0);
    if (g_old) load8(g_old, p, g0);
    const double x0 = x[p], y0 = y[p];
    double sxx = 0.0, sxy = 0.0, syy = 0.0;
    double sxq[4] = {0, 0, 0, 0}, syq[4] = {0, 0, 0, 0};
    // a row outside [0, nbr_offsets[n]] or running backwards is skipped and
    // reported, so that idx is only read inside its nbr_offsets[n] entries
    const int e0 = off[p], e1 = off[p + 1], nnz = off[n];
    if (e0 < 0 || e1 < e0 || e1 > nnz || e1 - e0 > LSKUM_MAX_DEGREE) {
        atomicOr(status, NA_BAD_OFFSETS);
        return;
    }
    for (int e = e0; e < e1; ++e) {
        const int i = idx[e];
        if (i < 0 || i >= n) {
            atomicOr(status, NA_BAD_INDEX);
            continue;
        }
        const double dx = x[i] - x0, dy = y[i] - y0;
        double qi[4];
        load4(q, i, qi);
        double gi[8];
        if (g_old) load8(g_old, i, gi);
        sxx += dx * dx;
        sxy += dx * dy;
        syy += dy * dy;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            double dq = qi[k] - q0[k];
            if (g_old) dq = dq - 0.5 * (dx * (gi[k] - g0[k]) + dy * (gi[4 + k] - g0[4 + k]));
            sxq[k] += dx * dq;
            syq[k] += dy * dq;
        }
    }
    const double inv = 1.0 / (sxx * syy - sxy * sxy);
    double out[8];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        out[k] = (syy * sxq[k] - sxy * syq[k]) * inv;
        out[4 + k] = (sxx * syq[k] - sxy * sxq[k]) * inv;
    }
    if (g_new) {
        store8(g_new, p, out);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            qx[k * n + p] = out[k];
            qy[k * n + p] = out[4 + k];
        }
    }
}

// Device address of the scratch array, looked up once per device with that
// device current (host code only sees a host-side stand-in for the symbol).
// The address belongs to the device's primary context: the library must not
// be used on a device after cudaDeviceReset there (the cached address would
// be stale).
static std::mutex g_noalloc_mutex;
static double *g_noalloc_ptr[128];

static cudaError_t noalloc_scratch(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = static_cast<double *>(ptr);
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

}  // namespace lskum

using namespace lskum;

static lskum_status na_fail(lskum_status st, const char *fmt, ...)
{
    char buf[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    set_global_error(buf);
    return st;
}

#define NA_CK(call)                                                                      \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return na_fail(LSKUM_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

extern "C" lskum_status lskum_q_derivatives_noalloc(int64_t n, const double *x, const double *y,
                                                    const int32_t *nbr_offsets, const int32_t *nbr_idx,
                                                    const double *U, double gamma, int inner_iters,
                                                    double *qx, double *qy, void *cuda_stream)
{
    set_global_error("");
    if (n < 1 || n > LSKUM_NOALLOC_MAX_POINTS)
        return na_fail(LSKUM_ERR_ARG, "n = %lld outside [1, %d], the size of the static scratch",
                       (long long)n, LSKUM_NOALLOC_MAX_POINTS);
    if (!x || !y || !nbr_offsets || !nbr_idx || !U || !qx || !qy)
        return na_fail(LSKUM_ERR_ARG, "a required pointer is NULL");
    if (inner_iters < 0 || inner_iters > 1000) return na_fail(LSKUM_ERR_ARG, "inner_iters out of range");
    if (!(gamma > 1.0)) return na_fail(LSKUM_ERR_ARG, "gamma must be > 1");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    double *base = nullptr;
    NA_CK(noalloc_scratch(&base));
    int *status = reinterpret_cast<int *>(base);
    double *q = base + kNoallocHeader;
    double *ga = q + 4 * n;
    double *gb = ga + 8 * n;
    // the status words must start at zero; q, ga, gb are written before read
    NA_CK(cudaMemsetAsync(status, 0, 2 * sizeof(int), s));
    Gas gas{};
    gas.gamma = gamma;
    gas.inv_gm1 = 1.0 / (gamma - 1.0);
    gas.hc = 0.5 * (gas.inv_gm1 + 1.0);
    gas.g14 = gamma == 1.4;
    const unsigned b256 = (unsigned)((n + 255) / 256), b128 = (unsigned)((n + 127) / 128);
    k_na_q<<<b256, 256, 0, s>>>(n, gas, U, q, status);
    NA_CK(cudaGetLastError());
    const double *g_old = nullptr;
    double *bufs[2] = {ga, gb};
    for (int it = 0; it <= inner_iters; ++it) {
        const bool last = it == inner_iters;
        double *g_new = last ? nullptr : bufs[it & 1];
        k_na_grad<<<b128, 128, 0, s>>>(n, x, y, nbr_offsets, nbr_idx, q, g_old, g_new, qx, qy, status);
        NA_CK(cudaGetLastError());
        g_old = g_new;
    }
    static thread_local int st_h[2];
    NA_CK(cudaMemcpyAsync(st_h, status, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    NA_CK(cudaStreamSynchronize(s));
    if (st_h[0] & NA_BAD_OFFSETS)
        return na_fail(LSKUM_ERR_CONNECTIVITY,
                       "nbr_offsets is not a CSR row array (a row runs backwards, leaves [0, nbr_offsets[n]] "
                       "or has more than %d entries)", LSKUM_MAX_DEGREE);
    if (st_h[0] & NA_BAD_INDEX) return na_fail(LSKUM_ERR_CONNECTIVITY, "a neighbour index is outside [0, n)");
    if (st_h[0] & NA_NONPHYSICAL) return na_fail(LSKUM_ERR_NONPHYSICAL, "a state has rho <= 0 or p <= 0");
    return LSKUM_OK;
}
