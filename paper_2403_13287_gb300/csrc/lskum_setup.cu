// Create-time kernels: sub-stencil split and least-squares weights (Sec. 2,
// E9, E11 and the N_x+-/N_y+- definition after E12), Morton renumbering,
// and the gathers/scatters between the caller's numbering and the internal one.
#include <cub/cub.cuh>

#include "lskum_device.cuh"
#include "lskum_kernels.h"

namespace lskum {

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Split and weights of one point.
// The split is bit-exact with a plain evaluation without fused multiply-add:
//   dx = x_i - x_0, dy = y_i - y_0, ds = dx ny - dy nx, dn = dx nx + dy ny
// x+ <=> ds < 0, x- <=> ds > 0, y+ <=> dn < 0, y- <=> dn > 0 (strict: an exact
// zero joins neither). Weights:
//   full stencil:  a_x = (Syy dx - Sxy dy)/det, a_y = (Sxx dy - Sxy dx)/det
//   sub-stencil k: w_s = (Snn_k ds - Ssn_k dn)/det_k, w_n = (Sss_k dn - Ssn_k ds)/det_k
// A sub-stencil that the point's residual does not use gets weight 0: far-field
// points use none, wall points drop y+ (no upwind points inside the body).
// Kinetic boundary mode (ioff != nullptr): a wall or far-field point also has
// the mirror images of its neighbours (CSR ioff/iidx/imask, built from the
// split of a first pass), at local offsets (ds, -dn) and global offsets
// (dx - 2 dn nx, dy - 2 dn ny); they enter every sum after the neighbours,
// and such a point uses all four sub-stencils.
__device__ __forceinline__ void edge_offsets(double2 P0, double2 N0, double2 Pi, double &dx, double &dy, double &ds,
                                             double &dn)
{
    dx = __dsub_rn(Pi.x, P0.x);
    dy = __dsub_rn(Pi.y, P0.y);
    ds = __dsub_rn(__dmul_rn(dx, N0.y), __dmul_rn(dy, N0.x));
    dn = __dadd_rn(__dmul_rn(dx, N0.x), __dmul_rn(dy, N0.y));
}

__device__ __forceinline__ void image_offsets(double2 N0, double &dx, double &dy, double &ds, double &dn)
{
    dx = __dsub_rn(dx, __dmul_rn(2.0 * dn, N0.x));
    dy = __dsub_rn(dy, __dmul_rn(2.0 * dn, N0.y));
    dn = -dn;
    (void)ds;
}

__global__ void __launch_bounds__(128) k_geometry(int64_t n, const double2 *__restrict__ xy,
                                                  const double2 *__restrict__ nrm,
                                                  const uint8_t *__restrict__ flag,
                                                  const int32_t *__restrict__ off,
                                                  const int32_t *__restrict__ idx,
                                                  uint8_t *__restrict__ mask, double2 *__restrict__ lsw,
                                                  double2 *__restrict__ fxw, double *__restrict__ dmin,
                                                  int *bad, ImageEdges im)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double2 P0 = xy[p];
    const double2 N0 = nrm[p];
    const uint8_t f = flag[p];
    double Sxx = 0.0, Sxy = 0.0, Syy = 0.0;
    double ss[4] = {0, 0, 0, 0}, sn[4] = {0, 0, 0, 0}, nn[4] = {0, 0, 0, 0};
    double d2min = 1.0 / 0.0;
    const int e0 = off[p], e1 = off[p + 1];
    const int i0 = im.off ? im.off[p] : 0, i1 = im.off ? im.off[p + 1] : 0;
    for (int e = e0; e < e1; ++e) {
        double dx, dy, ds, dn;
        edge_offsets(P0, N0, xy[idx[e]], dx, dy, ds, dn);
        uint8_t m = 0;
        if (ds < 0.0) m |= M_XPOS;
        if (ds > 0.0) m |= M_XNEG;
        if (dn < 0.0) m |= M_YPOS;
        if (dn > 0.0) m |= M_YNEG;
        mask[e] = m;
        Sxx += dx * dx;
        Sxy += dx * dy;
        Syy += dy * dy;
        const int ks = (m & M_XPOS) ? 0 : ((m & M_XNEG) ? 1 : -1);
        const int kn = (m & M_YPOS) ? 2 : ((m & M_YNEG) ? 3 : -1);
        if (ks >= 0) { ss[ks] += ds * ds; sn[ks] += ds * dn; nn[ks] += dn * dn; }
        if (kn >= 0) { ss[kn] += ds * ds; sn[kn] += ds * dn; nn[kn] += dn * dn; }
        const double d2 = dx * dx + dy * dy;
        d2min = d2 < d2min ? d2 : d2min;
    }
    for (int e = i0; e < i1; ++e) {
        double dx, dy, ds, dn;
        edge_offsets(P0, N0, xy[im.idx[e]], dx, dy, ds, dn);
        image_offsets(N0, dx, dy, ds, dn);
        const uint8_t m = im.mask[e];
        Sxx += dx * dx;
        Sxy += dx * dy;
        Syy += dy * dy;
        const int ks = (m & M_XPOS) ? 0 : ((m & M_XNEG) ? 1 : -1);
        const int kn = (m & M_YPOS) ? 2 : ((m & M_YNEG) ? 3 : -1);
        if (ks >= 0) { ss[ks] += ds * ds; sn[ks] += ds * dn; nn[ks] += dn * dn; }
        if (kn >= 0) { ss[kn] += ds * ds; sn[kn] += ds * dn; nn[kn] += dn * dn; }
    }
    dmin[p] = sqrt(d2min);
    const double detF = Sxx * Syy - Sxy * Sxy;
    bool good = detF > 1e-10 * Sxx * Syy;
    bool need[4];
    double det[4];
    const bool kinetic = im.kinetic && f != FLAG_INTERIOR;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        need[k] = (f == FLAG_INTERIOR) || kinetic || (f == FLAG_WALL && k != 2);
        det[k] = ss[k] * nn[k] - sn[k] * sn[k];
        if (need[k] && !(det[k] > 1e-10 * ss[k] * nn[k])) good = false;
    }
    if (!good) {
        atomicAdd(bad, 1);
        atomicMin(bad + 1, (int)p);
    }
    for (int e = e0; e < e1; ++e) {
        double dx, dy, ds, dn;
        edge_offsets(P0, N0, xy[idx[e]], dx, dy, ds, dn);
        const uint8_t m = mask[e];
        lsw[e] = make_double2((Syy * dx - Sxy * dy) / detF, (Sxx * dy - Sxy * dx) / detF);
        const int ks = (m & M_XPOS) ? 0 : ((m & M_XNEG) ? 1 : -1);
        const int kn = (m & M_YPOS) ? 2 : ((m & M_YNEG) ? 3 : -1);
        double ws = 0.0, wn = 0.0;
        if (ks >= 0 && need[ks]) ws = (nn[ks] * ds - sn[ks] * dn) / det[ks];
        if (kn >= 0 && need[kn]) wn = (ss[kn] * dn - sn[kn] * ds) / det[kn];
        fxw[e] = make_double2(ws, wn);
    }
    for (int e = i0; e < i1; ++e) {
        double dx, dy, ds, dn;
        edge_offsets(P0, N0, xy[im.idx[e]], dx, dy, ds, dn);
        image_offsets(N0, dx, dy, ds, dn);
        const uint8_t m = im.mask[e];
        im.lsw[e] = make_double2((Syy * dx - Sxy * dy) / detF, (Sxx * dy - Sxy * dx) / detF);
        const int ks = (m & M_XPOS) ? 0 : ((m & M_XNEG) ? 1 : -1);
        const int kn = (m & M_YPOS) ? 2 : ((m & M_YNEG) ? 3 : -1);
        double ws = 0.0, wn = 0.0;
        if (ks >= 0) ws = (nn[ks] * ds - sn[ks] * dn) / det[ks];
        if (kn >= 0) wn = (ss[kn] * dn - sn[kn] * ds) / det[kn];
        im.fxw[e] = make_double2(ws, wn);
        if (im.hd) im.hd[e] = make_double2(0.5 * dx, 0.5 * dy);
    }
}

cudaError_t launch_geometry(int64_t n, const double2 *xy, const double2 *nrm, const uint8_t *flag,
                            const int32_t *off, const int32_t *idx, uint8_t *mask, double2 *lsw,
                            double2 *fxw, double *dmin, int *bad, const ImageEdges &im, cudaStream_t s)
{
    k_geometry<<<nblk(n, 128), 128, 0, s>>>(n, xy, nrm, flag, off, idx, mask, lsw, fxw, dmin, bad, im);
    return cudaGetLastError();
}

// per edge (P_i - P_0)/2 (FP64 contexts): the E14 reconstruction and correction
// terms use it directly, two fused multiply-adds per component; hd_f (if not
// null) receives it rounded to FP32
__global__ void k_half_offsets(int64_t n, const double2 *__restrict__ xy, const int32_t *__restrict__ off,
                               const int32_t *__restrict__ idx, double2 *__restrict__ hd, float2 *__restrict__ hd_f)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double2 P0 = xy[p];
    for (int e = off[p]; e < off[p + 1]; ++e) {
        const double2 Pi = xy[idx[e]];
        const double2 h = make_double2(0.5 * (Pi.x - P0.x), 0.5 * (Pi.y - P0.y));
        hd[e] = h;
        if (hd_f) hd_f[e] = make_float2(__double2float_rn(h.x), __double2float_rn(h.y));
    }
}

cudaError_t launch_half_offsets(int64_t n, const double2 *xy, const int32_t *off, const int32_t *idx, double2 *hd,
                                float2 *hd_f, cudaStream_t s)
{
    k_half_offsets<<<nblk(n, 128), 128, 0, s>>>(n, xy, off, idx, hd, hd_f);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Morton (Z-order) renumbering: 32 bits per coordinate over the bounding box,
// stable radix sort of the 64-bit codes (equal codes keep input order).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t spread32(uint64_t v)
{
    v &= 0xffffffffull;
    v = (v | (v << 16)) & 0x0000ffff0000ffffull;
    v = (v | (v << 8)) & 0x00ff00ff00ff00ffull;
    v = (v | (v << 4)) & 0x0f0f0f0f0f0f0f0full;
    v = (v | (v << 2)) & 0x3333333333333333ull;
    v = (v | (v << 1)) & 0x5555555555555555ull;
    return v;
}

// host form of the same interleave, for keys built on the host (batches)
static uint64_t spread32_host(uint64_t v)
{
    v &= 0xffffffffull;
    v = (v | (v << 16)) & 0x0000ffff0000ffffull;
    v = (v | (v << 8)) & 0x00ff00ff00ff00ffull;
    v = (v | (v << 4)) & 0x0f0f0f0f0f0f0f0full;
    v = (v | (v << 2)) & 0x3333333333333333ull;
    v = (v | (v << 1)) & 0x5555555555555555ull;
    return v;
}

uint64_t morton_code_host(double x, double y, double xmin, double ymin, double scale, int bits)
{
    const double top = (double)((1ull << bits) - 1);
    double fx = (x - xmin) * scale, fy = (y - ymin) * scale;
    fx = fx < 0.0 ? 0.0 : (fx > top ? top : fx);
    fy = fy < 0.0 ? 0.0 : (fy > top ? top : fy);
    return spread32_host((uint64_t)fx) | (spread32_host((uint64_t)fy) << 1);
}

__global__ void k_iota32(int64_t n, int32_t *__restrict__ v)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) v[p] = (int32_t)p;
}

__global__ void k_morton(int64_t n, const double2 *__restrict__ xy, double xmin, double ymin,
                         double scale, uint64_t *__restrict__ code, int32_t *__restrict__ iota)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double2 P = xy[p];
    double fx = (P.x - xmin) * scale, fy = (P.y - ymin) * scale;
    fx = fx < 0.0 ? 0.0 : (fx > 4294967295.0 ? 4294967295.0 : fx);
    fy = fy < 0.0 ? 0.0 : (fy > 4294967295.0 ? 4294967295.0 : fy);
    code[p] = spread32((uint64_t)fx) | (spread32((uint64_t)fy) << 1);
    iota[p] = (int32_t)p;
}

cudaError_t morton_permutation(int64_t n, const double2 *xy, double xmin, double ymin, double scale,
                               int32_t *perm, cudaStream_t s)
{
    uint64_t *code = nullptr, *code_sorted = nullptr;
    int32_t *iota = nullptr;
    void *tmp = nullptr;
    size_t tmp_bytes = 0;
    cudaError_t err = cudaSuccess;
    do {
        if ((err = cudaMallocAsync(&code, n * sizeof(uint64_t), s)) != cudaSuccess) break;
        if ((err = cudaMallocAsync(&code_sorted, n * sizeof(uint64_t), s)) != cudaSuccess) break;
        if ((err = cudaMallocAsync(&iota, n * sizeof(int32_t), s)) != cudaSuccess) break;
        k_morton<<<nblk(n, 256), 256, 0, s>>>(n, xy, xmin, ymin, scale, code, iota);
        if ((err = cudaGetLastError()) != cudaSuccess) break;
        err = cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, code, code_sorted, iota, perm, (int)n, 0, 64, s);
        if (err != cudaSuccess) break;
        if ((err = cudaMallocAsync(&tmp, tmp_bytes, s)) != cudaSuccess) break;
        err = cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, code, code_sorted, iota, perm, (int)n, 0, 64, s);
    } while (0);
    if (tmp) cudaFreeAsync(tmp, s);
    if (iota) cudaFreeAsync(iota, s);
    if (code_sorted) cudaFreeAsync(code_sorted, s);
    if (code) cudaFreeAsync(code, s);
    return err;
}

// internal point `p` is input point perm[p]
__global__ void k_permute_points(int64_t n, const int32_t *__restrict__ perm, const double *__restrict__ x,
                                 const double *__restrict__ y, const double *__restrict__ nx,
                                 const double *__restrict__ ny, const int32_t *__restrict__ flags,
                                 double2 *__restrict__ xy, double2 *__restrict__ nrm,
                                 uint8_t *__restrict__ flag, int32_t *__restrict__ inv)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int32_t o = perm[p];
    xy[p] = make_double2(x[o], y[o]);
    nrm[p] = make_double2(nx[o], ny[o]);
    flag[p] = (uint8_t)flags[o];
    inv[o] = (int32_t)p;
}

cudaError_t launch_permute_points(int64_t n, const int32_t *perm, const double *x, const double *y,
                                  const double *nx, const double *ny, const int32_t *flags,
                                  double2 *xy, double2 *nrm, uint8_t *flag, int32_t *inv,
                                  cudaStream_t s)
{
    k_permute_points<<<nblk(n, 256), 256, 0, s>>>(n, perm, x, y, nx, ny, flags, xy, nrm, flag, inv);
    return cudaGetLastError();
}

__global__ void k_degrees(int64_t n, const int32_t *__restrict__ perm, const int32_t *__restrict__ off_in,
                          int32_t *__restrict__ deg)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int32_t o = perm[p];
    deg[p] = off_in[o + 1] - off_in[o];
}

// rows keep the caller's neighbour order, so per-point arithmetic does not
// depend on the numbering
__global__ void k_csr_fill(int64_t n, const int32_t *__restrict__ perm, const int32_t *__restrict__ inv,
                           const int32_t *__restrict__ off_in, const int32_t *__restrict__ idx_in,
                           const int32_t *__restrict__ off_out, int32_t *__restrict__ idx_out)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int32_t o = perm[p];
    const int32_t src = off_in[o], cnt = off_in[o + 1] - src, dst = off_out[p];
    for (int k = 0; k < cnt; ++k) idx_out[dst + k] = inv[idx_in[src + k]];
}

cudaError_t permute_csr(int64_t n, const int32_t *perm, const int32_t *inv, const int32_t *off_in,
                        const int32_t *idx_in, int32_t *off_out, int32_t *idx_out, cudaStream_t s)
{
    int32_t *deg = nullptr;
    void *tmp = nullptr;
    size_t tmp_bytes = 0;
    cudaError_t err = cudaSuccess;
    do {
        if ((err = cudaMallocAsync(&deg, n * sizeof(int32_t), s)) != cudaSuccess) break;
        k_degrees<<<nblk(n, 256), 256, 0, s>>>(n, perm, off_in, deg);
        if ((err = cudaGetLastError()) != cudaSuccess) break;
        if ((err = cudaMemsetAsync(off_out, 0, sizeof(int32_t), s)) != cudaSuccess) break;
        err = cub::DeviceScan::InclusiveSum(nullptr, tmp_bytes, deg, off_out + 1, (int)n, s);
        if (err != cudaSuccess) break;
        if ((err = cudaMallocAsync(&tmp, tmp_bytes, s)) != cudaSuccess) break;
        err = cub::DeviceScan::InclusiveSum(tmp, tmp_bytes, deg, off_out + 1, (int)n, s);
        if (err != cudaSuccess) break;
        k_csr_fill<<<nblk(n, 256), 256, 0, s>>>(n, perm, inv, off_in, idx_in, off_out, idx_out);
        err = cudaGetLastError();
    } while (0);
    if (tmp) cudaFreeAsync(tmp, s);
    if (deg) cudaFreeAsync(deg, s);
    return err;
}

// ---------------------------------------------------------------------------
// caller layout [4][n] (input numbering) <-> internal [n][4] (internal numbering)
// ---------------------------------------------------------------------------
__global__ void k_state_in(int64_t n, const int32_t *__restrict__ perm, const double *__restrict__ Uin,
                           double *__restrict__ U)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int64_t o = perm[p];
    double v[4] = {Uin[o], Uin[n + o], Uin[2 * n + o], Uin[3 * n + o]};
    store4(U, p, v);
}

__global__ void k_state_out(int64_t n, const int32_t *__restrict__ perm, const double *__restrict__ U,
                            double *__restrict__ Uout)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int64_t o = perm[p];
    double v[4];
    load4(U, p, v);
    Uout[o] = v[0]; Uout[n + o] = v[1]; Uout[2 * n + o] = v[2]; Uout[3 * n + o] = v[3];
}

__global__ void k_grad_out(int64_t n, const int32_t *__restrict__ perm, const double *__restrict__ qg,
                           double *__restrict__ qx, double *__restrict__ qy)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int64_t o = perm[p];
    double v[8];
    load8(qg, p, v);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        qx[k * n + o] = v[k];
        qy[k * n + o] = v[4 + k];
    }
}

__global__ void k_scalar_out(int64_t n, const int32_t *__restrict__ perm, const double *__restrict__ v,
                             double *__restrict__ out)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    out[perm[p]] = v[p];
}

// input CSR entry (o, k) is internal entry (inv[o], k)
__global__ void k_mask_out(int64_t n, const int32_t *__restrict__ inv, const int32_t *__restrict__ off_in,
                           const int32_t *__restrict__ off_int, const uint8_t *__restrict__ mask_int,
                           uint8_t *__restrict__ mask_in)
{
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n) return;
    const int32_t src = off_int[inv[o]], dst = off_in[o], cnt = off_in[o + 1] - dst;
    for (int k = 0; k < cnt; ++k) mask_in[dst + k] = mask_int[src + k];
}

__global__ void k_fill_state(int64_t n, double u0, double u1, double u2, double u3, double *__restrict__ U)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    double v[4] = {u0, u1, u2, u3};
    store4(U, p, v);
}

cudaError_t launch_state_in(int64_t n, const int32_t *perm, const double *Uin_cm, double *U_pm,
                            cudaStream_t s)
{
    k_state_in<<<nblk(n, 256), 256, 0, s>>>(n, perm, Uin_cm, U_pm);
    return cudaGetLastError();
}

cudaError_t launch_state_out(int64_t n, const int32_t *perm, const double *U_pm, double *Uout_cm,
                             cudaStream_t s)
{
    k_state_out<<<nblk(n, 256), 256, 0, s>>>(n, perm, U_pm, Uout_cm);
    return cudaGetLastError();
}

cudaError_t launch_grad_out(int64_t n, const int32_t *perm, const double *qg, double *qx_cm,
                            double *qy_cm, cudaStream_t s)
{
    k_grad_out<<<nblk(n, 256), 256, 0, s>>>(n, perm, qg, qx_cm, qy_cm);
    return cudaGetLastError();
}

cudaError_t launch_scalar_out(int64_t n, const int32_t *perm, const double *v, double *out,
                              cudaStream_t s)
{
    k_scalar_out<<<nblk(n, 256), 256, 0, s>>>(n, perm, v, out);
    return cudaGetLastError();
}

cudaError_t launch_mask_out(int64_t n, const int32_t *inv, const int32_t *off_in,
                            const int32_t *off_int, const uint8_t *mask_int, uint8_t *mask_in,
                            cudaStream_t s)
{
    k_mask_out<<<nblk(n, 256), 256, 0, s>>>(n, inv, off_in, off_int, mask_int, mask_in);
    return cudaGetLastError();
}

// free stream of each point's case
__global__ void k_fill_state_cases(int64_t n, const uint16_t *__restrict__ pcase,
                                   const double *__restrict__ case_uinf, double *__restrict__ U)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double *u = case_uinf + 4 * (int)pcase[p];
    double v[4] = {u[0], u[1], u[2], u[3]};
    store4(U, p, v);
}

cudaError_t launch_fill_state_cases(int64_t n, const uint16_t *pcase, const double *case_uinf, double *U,
                                    cudaStream_t s)
{
    k_fill_state_cases<<<nblk(n, 256), 256, 0, s>>>(n, pcase, case_uinf, U);
    return cudaGetLastError();
}

// sorting keys -> permutation (stable: equal keys keep input order)
cudaError_t sort_permutation(int64_t n, const uint64_t *keys, int32_t *perm, cudaStream_t s)
{
    uint64_t *sorted = nullptr;
    int32_t *iota = nullptr;
    void *tmp = nullptr;
    size_t tmp_bytes = 0;
    cudaError_t err = cudaSuccess;
    do {
        if ((err = cudaMallocAsync(&sorted, n * sizeof(uint64_t), s)) != cudaSuccess) break;
        if ((err = cudaMallocAsync(&iota, n * sizeof(int32_t), s)) != cudaSuccess) break;
        k_iota32<<<nblk(n, 256), 256, 0, s>>>(n, iota);
        if ((err = cudaGetLastError()) != cudaSuccess) break;
        err = cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, keys, sorted, iota, perm, (int)n, 0, 64, s);
        if (err != cudaSuccess) break;
        if ((err = cudaMallocAsync(&tmp, tmp_bytes, s)) != cudaSuccess) break;
        err = cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, keys, sorted, iota, perm, (int)n, 0, 64, s);
    } while (0);
    if (tmp) cudaFreeAsync(tmp, s);
    if (iota) cudaFreeAsync(iota, s);
    if (sorted) cudaFreeAsync(sorted, s);
    return err;
}

cudaError_t launch_fill_state(int64_t n, const double Uinf[4], double *U, cudaStream_t s)
{
    k_fill_state<<<nblk(n, 256), 256, 0, s>>>(n, Uinf[0], Uinf[1], Uinf[2], Uinf[3], U);
    return cudaGetLastError();
}

}  // namespace lskum
