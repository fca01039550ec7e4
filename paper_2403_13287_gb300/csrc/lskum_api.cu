// C ABI of the q-LSKUM hot path (include/lskum.h): context creation with CSR
// validation, renumbering and geometry; the pseudo-time loop of Algorithm 1
// (arXiv 2403.13287, Sec. 3); residual, derivative, time-step and force
// queries; state transfer.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "lskum.h"
#include "lskum_kernels.h"
#include "lskum_mixed.h"
#include "lskum_adjoint.h"

using namespace lskum;

// NVTX range over one library call (visible to Nsight tools; no cost without them)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

struct lskum_ctx {
    int64_t n = 0, nnz = 0, n_wall = 0;
    lskum_config cfg{};
    cudaStream_t stream = nullptr;
    std::string err;
    int64_t launches = 0;
    Gas gas{};
    std::vector<int32_t> perm_h;
    std::vector<void *> allocs;

    double2 *xy = nullptr, *nrm = nullptr;
    uint8_t *flag = nullptr, *mask = nullptr;
    double *dmin = nullptr;
    int32_t *off = nullptr, *idx = nullptr, *off_in = nullptr;
    double2 *lsw = nullptr, *fxw = nullptr, *hd = nullptr;
    float2 *hd_f = nullptr;  // FP64 contexts: hd in FP32, for the limiter's screening of d_m
    // kinetic boundary mode: mirror images of the neighbours of wall and
    // far-field points (CSR per internal point) and each case's free-stream q
    bool kinetic = false;
    int64_t nimg = 0;
    int32_t *ioff = nullptr, *iidx = nullptr;
    uint8_t *imask = nullptr;
    double2 *ilsw = nullptr, *ifxw = nullptr, *ihd = nullptr;
    double *qinf = nullptr;
    float *qinf_f = nullptr;
    float2 *ilsw_f = nullptr;
    float4 *igf = nullptr;
    int32_t *perm = nullptr, *inv = nullptr;
    int32_t *wall = nullptr;
    double *wall_ds = nullptr;

    double *U = nullptr, *Us = nullptr, *acc = nullptr, *Ubak = nullptr;
    // q and q-derivative buffers: double in the FP64 form, float in the mixed one
    void *q_cur = nullptr, *q_nxt = nullptr;
    void *qgA = nullptr, *qgB = nullptr;
    // second order: the first-order q-derivatives kept for the inner passes
    // ([n][8]) and the limiter's extremum measure ([n][4]), in the form's type
    void *qgG1 = nullptr, *qext = nullptr;
    bool mixed = false;
    int n_fp64_closure = 0;
    // mixed form: FP32 geometry view
    float2 *nrm_f = nullptr;
    float *dmin_f = nullptr;
    int32_t *slice_off = nullptr, *s_idx = nullptr;  // SELL-32 edge layout
    float2 *s_ga = nullptr;
    float4 *s_gf = nullptr, *gm = nullptr;
    double2 *s_fxw64 = nullptr;
    // staged flux variants: per tile the neighbours outside it, per slot its staged row
    int32_t *tile_off = nullptr, *tile_idx = nullptr;
    uint16_t *s_loc = nullptr;
    int64_t tile_overflow = 0;     // slots whose neighbour is beyond a tile's staging cap
    double *dt = nullptr, *Rt = nullptr, *Ut = nullptr, *Ucm = nullptr;
    double *norm_part = nullptr;   // residue_parts(n) values: a pair of sums per warp
    double *norm_chunk = nullptr;  // ncases * maxchunks chunk sums of the residue reduction
    int maxchunks = 1;
    double *res_dev = nullptr;     // residue history, [iteration][case]
    int res_cap = 0;               // iterations res_dev holds
    int *res_counter = nullptr;  // next entry of res_dev the residue kernel writes
    int *status = nullptr;

    // lskum_step replays one captured iteration (two for forward Euler, so
    // the q ping-pong ends where it began) as a CUDA graph; the graph bakes
    // in q_cur and res_dev, so one exec is kept per starting q buffer and
    // both are rebuilt when res_dev grows
    struct StepGraph {
        cudaGraphExec_t exec = nullptr;
        const void *q_start = nullptr;
        const double *res = nullptr;
        int iters = 0;
        int64_t launches = 0;
    };
    StepGraph graphs[2];
    cudaStream_t gstream = nullptr;  // capture stream (never the legacy default stream)
    bool graphs_off = false;

    // cases: a batch context solves several independent problems over the
    // disjoint union of their clouds; case c owns input and internal points
    // [case_start_h[c], case_start_h[c+1]) and wall entries
    // [case_wall_h[c], case_wall_h[c+1]); a single context is one case
    int ncases = 1;
    std::vector<int64_t> case_start_h, case_wall_h;
    std::vector<double> case_mach, case_aoa;
    int64_t *case_start = nullptr;   // device copy of case_start_h
    uint16_t *pcase = nullptr;       // per internal point: its case (batches only)
    double *case_uinf = nullptr;     // [ncases][4] (batches only)
    std::vector<uint16_t> case_of_input;  // create-time only

    // launch-shape variants of the mixed flux and q-derivative kernels
    int var_flux = 0, var_qgrad = 0;

    // residual VJP workspace (FP64, allocated on the first lskum_residual_vjp)
    bool vjp_ready = false;
    double *vq = nullptr, *vG = nullptr, *vRb = nullptr, *vqb = nullptr, *vgb = nullptr, *vgb2 = nullptr;
    double *vebar = nullptr;
    double2 *vwbar = nullptr, *vabar = nullptr, *vdbar = nullptr;
    int32_t *toff = nullptr, *tedge = nullptr, *tsrc = nullptr;
    double *vGlim = nullptr;      // [n][8] the limited last iterate (limiter_K > 0)
    double *vext = nullptr;       // [n][4] the limiter's extremum measure (limiter_K > 0)
    int32_t *vlidx = nullptr;     // [n][4] limiter reverse: the extreme neighbour's edge
    double *vlval = nullptr;      // [n][4] limiter reverse: its q cotangent
    double *vUacc = nullptr;      // [n][4] U cotangent being accumulated (internal order)
    double2 *vpxy = nullptr;      // [n] point cotangents of x, y gathered directly (forces)
    // update-step VJP (allocated on the first lskum_step_vjp): stage states,
    // stage residuals, their cotangents, dt and its cotangent
    bool svjp_ready = false;
    double *sR[4] = {}, *sU[3] = {}, *sRb[4] = {}, *sUb = nullptr, *sUin = nullptr, *sdt = nullptr, *sdtb = nullptr;
    double *fdsb = nullptr;       // forces VJP: cotangents of the arc-length weights
    // FP32 residual VJP (mixed contexts; allocated on the first such call)
    bool fvjp_ready = false;
    float *fq = nullptr, *fG = nullptr, *fRb = nullptr, *fqb = nullptr, *fgb = nullptr, *fgb2 = nullptr, *febar = nullptr;
    double *fbuf = nullptr;

    // kernel timing (lskum_profile): event pairs per kernel class, reused
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> timed[LSKUM_KERNEL_CLASSES];

    DevGeom geom() const
    {
        DevGeom g{};
        g.n = n; g.xy = xy; g.nrm = nrm; g.flag = flag; g.dmin = dmin;
        g.off = off; g.idx = idx; g.mask = mask; g.lsw = lsw; g.fxw = fxw; g.hd = hd; g.hd_f = hd_f;
        if (kinetic) {
            g.ioff = ioff; g.iidx = iidx; g.imask = imask; g.ilsw = ilsw; g.ifxw = ifxw; g.ihd = ihd;
            g.qinf = qinf; g.pcase = pcase;
        }
        return g;
    }

    MixedGeom mgeom() const
    {
        MixedGeom g{};
        g.n = n; g.nrm = nrm_f; g.flag = flag; g.dmin = dmin_f; g.off = off;
        g.slice_off = slice_off; g.sidx = s_idx; g.ga = s_ga; g.gm = gm; g.gf = s_gf; g.fxw64 = s_fxw64;
        g.tile_off = tile_off; g.tile_idx = tile_idx; g.sloc = s_loc;
        if (kinetic) {
            g.ioff = ioff; g.iidx = iidx; g.imask = imask; g.ilsw = ilsw_f; g.igf = igf; g.ifxw64 = ifxw;
            g.qinf = qinf_f; g.pcase = pcase;
        }
        return g;
    }
};

static thread_local std::string g_create_error;

namespace lskum {
// error text for calls without a context (lskum_last_error(NULL))
void set_global_error(const char *msg) { g_create_error = msg; }
}  // namespace lskum

static lskum_status fail(lskum_ctx *c, lskum_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    else g_create_error = buf;
    return st;
}

#define CK(c, call)                                                                             \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return fail((c), e_ == cudaErrorMemoryAllocation ? LSKUM_ERR_OOM : LSKUM_ERR_CUDA,  \
                        "%s failed: %s", #call, cudaGetErrorString(e_));                         \
    } while (0)

#define LAUNCH(c, call)                                                                         \
    do {                                                                                        \
        (c)->launches++;                                                                        \
        CK(c, call);                                                                            \
    } while (0)

// evaluates a launch; false (and r set) on failure
#define LAUNCH_OK(c, call, r)                                                                   \
    ([&]() -> bool {                                                                            \
        (c)->launches++;                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ == cudaSuccess) return true;                                                     \
        (r) = fail((c), LSKUM_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));         \
        return false;                                                                           \
    }())

static cudaError_t next_event(lskum_ctx *c, cudaEvent_t *ev)
{
    if (c->ev_used == c->ev_pool.size()) {
        cudaEvent_t e;
        cudaError_t err = cudaEventCreate(&e);
        if (err != cudaSuccess) return err;
        c->ev_pool.push_back(e);
    }
    *ev = c->ev_pool[c->ev_used++];
    return cudaSuccess;
}

// launch of a timed kernel class: bracketed by events while profiling
#define TIMED_LAUNCH(c, cls, call)                                                              \
    do {                                                                                        \
        cudaEvent_t e0_ = nullptr, e1_ = nullptr;                                               \
        if ((c)->profiling) {                                                                   \
            CK(c, next_event(c, &e0_));                                                         \
            CK(c, next_event(c, &e1_));                                                         \
            CK(c, cudaEventRecord(e0_, (c)->stream));                                           \
        }                                                                                       \
        LAUNCH(c, call);                                                                        \
        if ((c)->profiling) {                                                                   \
            CK(c, cudaEventRecord(e1_, (c)->stream));                                           \
            (c)->timed[cls].push_back({e0_, e1_});                                              \
        }                                                                                       \
    } while (0)

template <typename T>
static cudaError_t dalloc(lskum_ctx *c, T **p, size_t count)
{
    void *v = nullptr;
    cudaError_t e = cudaMalloc(&v, std::max<size_t>(count, 1) * sizeof(T));
    if (e == cudaSuccess) {
        c->allocs.push_back(v);
        *p = static_cast<T *>(v);
    }
    return e;
}

static void free_all(lskum_ctx *c)
{
    for (void *p : c->allocs) cudaFree(p);
    c->allocs.clear();
}

static void freestream(double gamma, double mach, double aoa_deg, double U[4])
{
    const double a = aoa_deg * 3.14159265358979323846 / 180.0;
    const double rho = 1.0, u = mach * cos(a), v = mach * sin(a), p = 1.0 / gamma;
    U[0] = rho;
    U[1] = rho * u;
    U[2] = rho * v;
    U[3] = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v);
}

static lskum_status validate_csr(int64_t n, const int32_t *off, const int32_t *idx, std::string &msg)
{
    char buf[256];
    if (off[0] != 0) { msg = "nbr_offsets[0] != 0"; return LSKUM_ERR_CONNECTIVITY; }
    std::vector<int32_t> row;
    for (int64_t p = 0; p < n; ++p) {
        const int64_t a = off[p], b = off[p + 1];
        if (b < a) {
            snprintf(buf, sizeof buf, "nbr_offsets decreases at point %lld", (long long)p);
            msg = buf; return LSKUM_ERR_CONNECTIVITY;
        }
        if (b - a > LSKUM_MAX_DEGREE) {
            snprintf(buf, sizeof buf, "point %lld has %lld neighbours (max %d)", (long long)p,
                     (long long)(b - a), LSKUM_MAX_DEGREE);
            msg = buf; return LSKUM_ERR_CONNECTIVITY;
        }
        row.assign(idx + a, idx + b);
        for (int32_t i : row) {
            if (i < 0 || i >= n) {
                snprintf(buf, sizeof buf, "point %lld has neighbour index %d out of range", (long long)p, i);
                msg = buf; return LSKUM_ERR_CONNECTIVITY;
            }
            if (i == p) {
                snprintf(buf, sizeof buf, "point %lld lists itself as a neighbour", (long long)p);
                msg = buf; return LSKUM_ERR_CONNECTIVITY;
            }
        }
        std::sort(row.begin(), row.end());
        for (size_t k = 1; k < row.size(); ++k)
            if (row[k] == row[k - 1]) {
                snprintf(buf, sizeof buf, "point %lld lists neighbour %d twice", (long long)p, row[k]);
                msg = buf; return LSKUM_ERR_CONNECTIVITY;
            }
    }
    return LSKUM_OK;
}

extern "C" const char *lskum_last_error(const lskum_ctx *ctx)
{
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

extern "C" int64_t lskum_launch_count(const lskum_ctx *ctx) { return ctx ? ctx->launches : 0; }

extern "C" void lskum_destroy(lskum_ctx *ctx)
{
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    for (auto &g : ctx->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    if (ctx->gstream) cudaStreamDestroy(ctx->gstream);
    free_all(ctx);
    delete ctx;
}

// q-variables of an internal-layout state U ([n][4]) into qdst, in the
// context's precision
static lskum_status refresh_q(lskum_ctx *c, const double *U, void *qdst)
{
    if (c->mixed) LAUNCH(c, launch_q_from_U_mixed(c->n, c->gas, U, (float *)qdst, c->status, c->stream));
    else LAUNCH(c, launch_q_from_U(c->n, c->gas, U, (double *)qdst, c->status, c->stream));
    return LSKUM_OK;
}

// Reverse Cuthill-McKee numbering of the stencil graph (E. Cuthill and
// J. McKee, Proc. 24th ACM National Conference, 1969; reversed as in A.
// George, 1971): per connected component, breadth-first from a
// pseudo-peripheral point (George-Liu: repeat from a farthest point of
// smallest degree while the eccentricity grows), neighbours visited by
// increasing degree, ties by index; each component's order is then reversed
// in place, so components keep the order of their smallest point (a batch's
// cases stay contiguous and in case order). The graph is the CSR relation
// made symmetric. perm[k] = input index of the k-th point.
static void rcm_permutation(int64_t n, const int32_t *off, const int32_t *idx, std::vector<int32_t> &perm)
{
    // symmetric adjacency
    std::vector<int64_t> cnt(n + 1, 0);
    for (int64_t p = 0; p < n; ++p)
        for (int32_t e = off[p]; e < off[p + 1]; ++e) {
            ++cnt[p + 1];
            ++cnt[idx[e] + 1];
        }
    for (int64_t p = 0; p < n; ++p) cnt[p + 1] += cnt[p];
    std::vector<int32_t> adj(cnt[n]);
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    for (int64_t p = 0; p < n; ++p)
        for (int32_t e = off[p]; e < off[p + 1]; ++e) {
            adj[fill[p]++] = idx[e];
            adj[fill[idx[e]]++] = (int32_t)p;
        }
    std::vector<int32_t> deg(n);
    for (int64_t p = 0; p < n; ++p) {
        std::sort(adj.begin() + cnt[p], adj.begin() + cnt[p + 1]);
        const auto last = std::unique(adj.begin() + cnt[p], adj.begin() + cnt[p + 1]);
        deg[p] = (int32_t)(last - (adj.begin() + cnt[p]));
    }
    std::vector<int32_t> level(n, -1), order;
    order.reserve(n);
    std::vector<int32_t> nb;
    // breadth-first from `root`, neighbours by (degree, index); appends to out,
    // marks level; returns the last level's size and a smallest-degree point on it
    auto bfs = [&](int32_t root, std::vector<int32_t> &out, std::vector<int32_t> &lv, int32_t *far) {
        const size_t start = out.size();
        lv[root] = 0;
        out.push_back(root);
        for (size_t h = start; h < out.size(); ++h) {
            const int32_t u = out[h];
            nb.assign(adj.begin() + cnt[u], adj.begin() + cnt[u] + deg[u]);
            std::sort(nb.begin(), nb.end(), [&](int32_t a, int32_t b) {
                return deg[a] != deg[b] ? deg[a] < deg[b] : a < b;
            });
            for (int32_t v : nb)
                if (lv[v] < 0) {
                    lv[v] = lv[u] + 1;
                    out.push_back(v);
                }
        }
        const int32_t depth = lv[out.back()];
        int32_t best = out.back();
        for (size_t h = start; h < out.size(); ++h) {
            const int32_t v = out[h];
            if (lv[v] == depth && (deg[v] < deg[best] || (deg[v] == deg[best] && v < best))) best = v;
        }
        *far = best;
        return depth;
    };
    std::vector<int32_t> scratch, lv2(n, -1);
    for (int64_t s0 = 0; s0 < n; ++s0) {
        if (level[s0] >= 0) continue;
        // pseudo-peripheral root of this component
        int32_t root = (int32_t)s0, far = root;
        scratch.clear();
        int32_t ecc = bfs(root, scratch, lv2, &far);
        for (int it = 0; it < 8; ++it) {
            for (int32_t v : scratch) lv2[v] = -1;
            std::vector<int32_t> tmp;
            int32_t far2 = far;
            const int32_t e2 = bfs(far, tmp, lv2, &far2);
            if (e2 <= ecc) {
                for (int32_t v : tmp) lv2[v] = -1;
                break;
            }
            root = far;
            ecc = e2;
            scratch.swap(tmp);
            far = far2;
        }
        for (int32_t v : scratch) lv2[v] = -1;
        const size_t a = order.size();
        int32_t dummy;
        bfs(root, order, level, &dummy);
        std::reverse(order.begin() + a, order.end());
    }
    perm.assign(order.begin(), order.end());
}

// Staged flux variants: for every tile of kTile consecutive points (internal
// numbering), the neighbours outside the tile, each once and in increasing
// order, and for every SELL slot the row of its neighbour in the tile's
// staged block: the tile's own points are rows 0..kTile-1, its first
// kHaloCap outside neighbours rows kTile.., a neighbour beyond that cap is
// kSlotGlobal (read from global memory). Padding slots get the point's own row.
static lskum_status build_tiles(lskum_ctx *c, const std::vector<int32_t> &off_h, const std::vector<int32_t> &so)
{
    const int64_t n = c->n, nnz = off_h[n];
    const cudaStream_t s = c->stream;
    std::vector<int32_t> idx_h(std::max<int64_t>(nnz, 1));
    std::vector<uint8_t> mask_h(std::max<int64_t>(nnz, 1));
    if (nnz > 0) {
        CK(c, cudaMemcpyAsync(idx_h.data(), c->idx, nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        CK(c, cudaMemcpyAsync(mask_h.data(), c->mask, nnz * sizeof(uint8_t), cudaMemcpyDeviceToHost, s));
    }
    CK(c, cudaStreamSynchronize(s));
    const int64_t ntiles = (n + kTile - 1) / kTile;
    const int64_t nslot = std::max<int32_t>(so.back(), 1);
    std::vector<int32_t> toff(ntiles + 1, 0), tidx;
    tidx.reserve((size_t)ntiles * 96);
    std::vector<uint16_t> sloc(nslot, 0);
    std::vector<int32_t> outside;
    int64_t overflow = 0;
    for (int64_t t = 0; t < ntiles; ++t) {
        const int64_t p0 = t * kTile, p1 = std::min<int64_t>(n, p0 + kTile);
        outside.clear();
        for (int64_t p = p0; p < p1; ++p)
            for (int32_t e = off_h[p]; e < off_h[p + 1]; ++e)
                if (idx_h[e] < p0 || idx_h[e] >= p1) outside.push_back(idx_h[e]);
        std::sort(outside.begin(), outside.end());
        outside.erase(std::unique(outside.begin(), outside.end()), outside.end());
        if ((int64_t)toff[t] + (int64_t)outside.size() > 0x7fffffff)
            return fail(c, LSKUM_ERR_ARG, "too many stencil entries for the staged tiles");
        toff[t + 1] = toff[t] + (int32_t)outside.size();
        tidx.insert(tidx.end(), outside.begin(), outside.end());
        for (int64_t p = p0; p < p1; ++p) {
            const int64_t base = so[p >> 5] + (p & 31);
            const int deg = off_h[p + 1] - off_h[p];
            const int depth = (so[(p >> 5) + 1] - so[p >> 5]) >> 5;
            for (int k = 0; k < depth; ++k) {
                uint16_t v = (uint16_t)(p - p0);
                if (k < deg) {
                    const int32_t e = off_h[p] + k, i = idx_h[e];
                    int row;
                    if (i >= p0 && i < p1) {
                        row = (int)(i - p0);
                    } else {
                        const int64_t r = std::lower_bound(outside.begin(), outside.end(), i) - outside.begin();
                        row = r < kHaloCap ? kTile + (int)r : kSlotGlobal;
                        overflow += r >= kHaloCap;
                    }
                    v = (uint16_t)(row | ((mask_h[e] & 0xf) << 12));
                }
                sloc[base + 32 * k] = v;
            }
        }
    }
    c->tile_overflow = overflow;
    CK(c, dalloc(c, &c->tile_off, ntiles + 1));
    CK(c, dalloc(c, &c->tile_idx, std::max<int64_t>((int64_t)tidx.size(), 1)));
    CK(c, dalloc(c, &c->s_loc, nslot));
    CK(c, cudaMemcpyAsync(c->tile_off, toff.data(), (ntiles + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    if (!tidx.empty())
        CK(c, cudaMemcpyAsync(c->tile_idx, tidx.data(), tidx.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    CK(c, cudaMemcpyAsync(c->s_loc, sloc.data(), nslot * sizeof(uint16_t), cudaMemcpyHostToDevice, s));
    CK(c, cudaStreamSynchronize(s));
    return LSKUM_OK;
}

static lskum_status create_impl(lskum_ctx *c, const double *x, const double *y, const double *nx,
                                const double *ny, const int32_t *flags, const int32_t *nbr_offsets,
                                const int32_t *nbr_idx, const int32_t *wall_order)
{
    NvtxRange nvtx_("lskum_create");
    const int64_t n = c->n, nnz = c->nnz;
    cudaStream_t s = c->stream;
    // input-order copies
    double *dx = nullptr, *dy = nullptr, *dnx = nullptr, *dny = nullptr;
    int32_t *dflags = nullptr, *didx_in = nullptr;
    CK(c, dalloc(c, &dx, n));
    CK(c, dalloc(c, &dy, n));
    CK(c, dalloc(c, &dnx, n));
    CK(c, dalloc(c, &dny, n));
    CK(c, dalloc(c, &dflags, n));
    CK(c, dalloc(c, &didx_in, nnz));
    CK(c, dalloc(c, &c->off_in, n + 1));
    CK(c, cudaMemcpyAsync(dx, x, n * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(c, cudaMemcpyAsync(dy, y, n * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(c, cudaMemcpyAsync(dnx, nx, n * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(c, cudaMemcpyAsync(dny, ny, n * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(c, cudaMemcpyAsync(dflags, flags, n * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    CK(c, cudaMemcpyAsync(didx_in, nbr_idx, nnz * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    CK(c, cudaMemcpyAsync(c->off_in, nbr_offsets, (n + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, s));

    CK(c, dalloc(c, &c->xy, n));
    CK(c, dalloc(c, &c->nrm, n));
    CK(c, dalloc(c, &c->flag, n));
    CK(c, dalloc(c, &c->dmin, n));
    CK(c, dalloc(c, &c->perm, n));
    CK(c, dalloc(c, &c->inv, n));
    CK(c, dalloc(c, &c->off, n + 1));
    CK(c, dalloc(c, &c->idx, nnz));
    CK(c, dalloc(c, &c->mask, nnz));
    CK(c, dalloc(c, &c->lsw, nnz));
    CK(c, dalloc(c, &c->fxw, nnz));

    // numbering (a batch keeps each case's points together, in case order)
    if (c->cfg.reorder == 1 && c->ncases > 1) {
        std::vector<uint64_t> keys(n);
        for (int k = 0; k < c->ncases; ++k) {
            const int64_t a = c->case_start_h[k], b = c->case_start_h[k + 1];
            double xmin = x[a], xmax = x[a], ymin = y[a], ymax = y[a];
            for (int64_t p = a + 1; p < b; ++p) {
                xmin = std::min(xmin, x[p]); xmax = std::max(xmax, x[p]);
                ymin = std::min(ymin, y[p]); ymax = std::max(ymax, y[p]);
            }
            const double ext = std::max(std::max(xmax - xmin, ymax - ymin), 1e-300);
            const double scale = 16777215.0 / ext;  // 24 bits per coordinate below the case bits
            for (int64_t p = a; p < b; ++p)
                keys[p] = ((uint64_t)k << 48) | morton_code_host(x[p], y[p], xmin, ymin, scale, 24);
        }
        uint64_t *keys_d = nullptr;
        CK(c, cudaMallocAsync(&keys_d, n * sizeof(uint64_t), s));
        CK(c, cudaMemcpyAsync(keys_d, keys.data(), n * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
        c->launches += 3;
        CK(c, sort_permutation(n, keys_d, c->perm, s));
        CK(c, cudaFreeAsync(keys_d, s));
        CK(c, cudaStreamSynchronize(s));
    } else if (c->cfg.reorder == 2) {
        std::vector<int32_t> pr;
        rcm_permutation(n, nbr_offsets, nbr_idx, pr);
        CK(c, cudaMemcpyAsync(c->perm, pr.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        CK(c, cudaStreamSynchronize(s));
    } else if (c->cfg.reorder == 1) {
        double xmin = x[0], xmax = x[0], ymin = y[0], ymax = y[0];
        for (int64_t p = 1; p < n; ++p) {
            xmin = std::min(xmin, x[p]); xmax = std::max(xmax, x[p]);
            ymin = std::min(ymin, y[p]); ymax = std::max(ymax, y[p]);
        }
        const double ext = std::max(std::max(xmax - xmin, ymax - ymin), 1e-300);
        const double scale = 4294967295.0 / ext;
        // the Morton kernel reads coordinates in input order
        double2 *xy_in = nullptr;
        CK(c, cudaMallocAsync(&xy_in, n * sizeof(double2), s));
        std::vector<double2> tmp(n);
        for (int64_t p = 0; p < n; ++p) tmp[p] = make_double2(x[p], y[p]);
        CK(c, cudaMemcpyAsync(xy_in, tmp.data(), n * sizeof(double2), cudaMemcpyHostToDevice, s));
        c->launches += 2;
        CK(c, morton_permutation(n, xy_in, xmin, ymin, scale, c->perm, s));
        CK(c, cudaFreeAsync(xy_in, s));
        CK(c, cudaStreamSynchronize(s));
    } else {
        std::vector<int32_t> iota(n);
        for (int64_t p = 0; p < n; ++p) iota[p] = (int32_t)p;
        CK(c, cudaMemcpyAsync(c->perm, iota.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        CK(c, cudaStreamSynchronize(s));
    }
    LAUNCH(c, launch_permute_points(n, c->perm, dx, dy, dnx, dny, dflags, c->xy, c->nrm, c->flag, c->inv, s));
    c->launches += 2;
    CK(c, permute_csr(n, c->perm, c->inv, c->off_in, didx_in, c->off, c->idx, s));

    int *bad = nullptr;
    CK(c, dalloc(c, &bad, 2));
    const int bad_init[2] = {0, 0x7fffffff};
    CK(c, cudaMemcpyAsync(bad, bad_init, sizeof bad_init, cudaMemcpyHostToDevice, s));
    LAUNCH(c, launch_geometry(n, c->xy, c->nrm, c->flag, c->off, c->idx, c->mask, c->lsw, c->fxw, c->dmin, bad,
                              ImageEdges{}, s));
    if (c->kinetic) {
        // the mirror images: one per neighbour off the tangent line (a split
        // bit in y) of each wall and far-field point, x+- kept, y+- swapped
        std::vector<int32_t> off_h(n + 1), idx_h(nnz);
        std::vector<uint8_t> mask_h(std::max<int64_t>(nnz, 1)), flag_h(n);
        CK(c, cudaMemcpyAsync(off_h.data(), c->off, (n + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        CK(c, cudaMemcpyAsync(idx_h.data(), c->idx, nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        CK(c, cudaMemcpyAsync(mask_h.data(), c->mask, nnz, cudaMemcpyDeviceToHost, s));
        CK(c, cudaMemcpyAsync(flag_h.data(), c->flag, n, cudaMemcpyDeviceToHost, s));
        CK(c, cudaStreamSynchronize(s));
        std::vector<int32_t> ioff_h(n + 1, 0), iidx_h;
        std::vector<uint8_t> imask_h;
        for (int64_t p = 0; p < n; ++p) {
            const uint8_t f = flag_h[p] & 3;
            if (f == FLAG_WALL || f == FLAG_FARFIELD) {
                for (int32_t e = off_h[p]; e < off_h[p + 1]; ++e) {
                    const uint8_t m = mask_h[e];
                    if (!(m & (M_YPOS | M_YNEG))) continue;
                    iidx_h.push_back(idx_h[e]);
                    imask_h.push_back((uint8_t)((m & (M_XPOS | M_XNEG)) | ((m & M_YPOS) ? M_YNEG : 0) |
                                                ((m & M_YNEG) ? M_YPOS : 0) |
                                                (f == FLAG_WALL ? M_IMG_WALL : M_IMG_FAR)));
                }
            }
            ioff_h[p + 1] = (int32_t)iidx_h.size();
        }
        c->nimg = (int64_t)iidx_h.size();
        const int64_t ni = std::max<int64_t>(c->nimg, 1);
        CK(c, dalloc(c, &c->ioff, n + 1));
        CK(c, dalloc(c, &c->iidx, ni));
        CK(c, dalloc(c, &c->imask, ni));
        CK(c, dalloc(c, &c->ilsw, ni));
        CK(c, dalloc(c, &c->ifxw, ni));
        CK(c, dalloc(c, &c->ihd, ni));
        CK(c, cudaMemcpyAsync(c->ioff, ioff_h.data(), (n + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        if (c->nimg > 0) {
            CK(c, cudaMemcpyAsync(c->iidx, iidx_h.data(), c->nimg * sizeof(int32_t), cudaMemcpyHostToDevice, s));
            CK(c, cudaMemcpyAsync(c->imask, imask_h.data(), c->nimg, cudaMemcpyHostToDevice, s));
        }
        // the weights again, now over the augmented stencils (the split of the
        // first pass is recomputed identically)
        CK(c, cudaMemcpyAsync(bad, bad_init, sizeof bad_init, cudaMemcpyHostToDevice, s));
        ImageEdges im;
        im.off = c->ioff; im.idx = c->iidx; im.mask = c->imask;
        im.lsw = c->ilsw; im.fxw = c->ifxw; im.hd = c->ihd; im.kinetic = 1;
        LAUNCH(c, launch_geometry(n, c->xy, c->nrm, c->flag, c->off, c->idx, c->mask, c->lsw, c->fxw, c->dmin,
                                  bad, im, s));
    }
    if (!c->mixed) {
        CK(c, dalloc(c, &c->hd, std::max<int64_t>(nnz, 1)));
        CK(c, dalloc(c, &c->hd_f, std::max<int64_t>(nnz, 1)));
        LAUNCH(c, launch_half_offsets(n, c->xy, c->off, c->idx, c->hd, c->hd_f, s));
    }
    int bad_h[2];
    CK(c, cudaMemcpyAsync(bad_h, bad, sizeof bad_h, cudaMemcpyDeviceToHost, s));
    c->perm_h.resize(n);
    CK(c, cudaMemcpyAsync(c->perm_h.data(), c->perm, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(c, cudaStreamSynchronize(s));
    if (bad_h[0] > 0) {
        const int32_t p_in = c->perm_h[bad_h[1]];
        return fail(c, LSKUM_ERR_DEGENERATE_STENCIL,
                    "%d point(s) have a singular least-squares stencil; first: point %d (flag %d)",
                    bad_h[0], p_in, flags[p_in]);
    }

    // wall contour (internal numbering) and its arc-length weights
    std::vector<int32_t> inv_h(n);
    for (int64_t p = 0; p < n; ++p) inv_h[c->perm_h[p]] = (int32_t)p;
    const int64_t nw = c->n_wall;
    std::vector<int32_t> wall_h(std::max<int64_t>(nw, 1));
    std::vector<double> ds_h(std::max<int64_t>(nw, 1));
    for (int k = 0; k < c->ncases; ++k) {
        // each case's contour is closed on itself
        const int64_t w0 = c->case_wall_h[k], m = c->case_wall_h[k + 1] - w0;
        for (int64_t j = 0; j < m; ++j) {
            const int32_t p = wall_order[w0 + j], pn = wall_order[w0 + (j + 1) % m],
                          pp = wall_order[w0 + (j + m - 1) % m];
            const double dn = sqrt((x[pn] - x[p]) * (x[pn] - x[p]) + (y[pn] - y[p]) * (y[pn] - y[p]));
            const double dp = sqrt((x[p] - x[pp]) * (x[p] - x[pp]) + (y[p] - y[pp]) * (y[p] - y[pp]));
            ds_h[w0 + j] = 0.5 * (dn + dp);
            wall_h[w0 + j] = inv_h[p];
        }
    }
    CK(c, dalloc(c, &c->wall, std::max<int64_t>(nw, 1)));
    CK(c, dalloc(c, &c->wall_ds, std::max<int64_t>(nw, 1)));
    CK(c, dalloc(c, &c->fbuf, nw + 2 * c->ncases));
    // case tables
    CK(c, dalloc(c, &c->case_start, c->ncases + 1));
    CK(c, cudaMemcpyAsync(c->case_start, c->case_start_h.data(), (c->ncases + 1) * sizeof(int64_t),
                          cudaMemcpyHostToDevice, s));
    if (c->ncases > 1) {
        std::vector<uint16_t> pc(n);
        for (int64_t p = 0; p < n; ++p) pc[p] = c->case_of_input[c->perm_h[p]];
        std::vector<double> ui(4 * c->ncases);
        for (int k = 0; k < c->ncases; ++k)
            freestream(c->cfg.gamma, c->case_mach[k], c->case_aoa[k], ui.data() + 4 * k);
        CK(c, dalloc(c, &c->pcase, n));
        CK(c, dalloc(c, &c->case_uinf, 4 * c->ncases));
        CK(c, cudaMemcpyAsync(c->pcase, pc.data(), n * sizeof(uint16_t), cudaMemcpyHostToDevice, s));
        CK(c, cudaMemcpyAsync(c->case_uinf, ui.data(), 4 * c->ncases * sizeof(double), cudaMemcpyHostToDevice, s));
        CK(c, cudaStreamSynchronize(s));
        std::vector<uint16_t>().swap(c->case_of_input);
    }
    if (nw > 0) {
        CK(c, cudaMemcpyAsync(c->wall, wall_h.data(), nw * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        CK(c, cudaMemcpyAsync(c->wall_ds, ds_h.data(), nw * sizeof(double), cudaMemcpyHostToDevice, s));
    }

    // state and work buffers
    CK(c, dalloc(c, &c->U, 4 * n));
    CK(c, dalloc(c, &c->Us, 4 * n));
    CK(c, dalloc(c, &c->acc, 4 * n));
    CK(c, dalloc(c, &c->Ubak, 4 * n));
    const size_t qbytes = c->mixed ? sizeof(float) : sizeof(double);
    {
        char *b = nullptr;
        CK(c, dalloc(c, &b, 2 * 4 * n * qbytes));
        c->q_cur = b;
        c->q_nxt = b + 4 * n * qbytes;
        CK(c, dalloc(c, &b, 2 * 8 * n * qbytes));
        c->qgA = b;
        c->qgB = b + 8 * n * qbytes;
    }
    if (c->cfg.order == 2) {
        char *b = nullptr;
        CK(c, dalloc(c, &b, 12 * n * qbytes));
        c->qgG1 = b;
        c->qext = b + 8 * n * qbytes;
    }
    if (c->mixed) {
        // FP32 geometry in CSR order, then scattered into the SELL-32 layout
        CK(c, dalloc(c, &c->nrm_f, n));
        CK(c, dalloc(c, &c->dmin_f, n));
        float2 *dxy = nullptr, *lsw = nullptr, *fxw = nullptr;
        CK(c, cudaMallocAsync(&dxy, std::max<int64_t>(nnz, 1) * sizeof(float2), s));
        CK(c, cudaMallocAsync(&lsw, std::max<int64_t>(nnz, 1) * sizeof(float2), s));
        CK(c, cudaMallocAsync(&fxw, std::max<int64_t>(nnz, 1) * sizeof(float2), s));
        int *cnt = nullptr;
        CK(c, dalloc(c, &cnt, 1));
        CK(c, cudaMemsetAsync(cnt, 0, sizeof(int), s));
        CK(c, dalloc(c, &c->gm, n));
        if (c->kinetic) {
            CK(c, dalloc(c, &c->ilsw_f, std::max<int64_t>(c->nimg, 1)));
            CK(c, dalloc(c, &c->igf, std::max<int64_t>(c->nimg, 1)));
        }
        LAUNCH(c, launch_mixed_prep(c->geom(), c->flag, c->nrm_f, c->dmin_f, c->gm, dxy, lsw, fxw, c->ilsw_f, c->igf,
                                    cnt, s));
        CK(c, cudaMemcpyAsync(&c->n_fp64_closure, cnt, sizeof(int), cudaMemcpyDeviceToHost, s));
        std::vector<int32_t> off_h(n + 1);
        CK(c, cudaMemcpyAsync(off_h.data(), c->off, (n + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        CK(c, cudaStreamSynchronize(s));
        const int64_t nslices = (n + 31) / 32;
        std::vector<int32_t> so(nslices + 1, 0);
        for (int64_t sl = 0; sl < nslices; ++sl) {
            int depth = 0;
            for (int64_t p = 32 * sl; p < std::min<int64_t>(n, 32 * sl + 32); ++p)
                depth = std::max(depth, off_h[p + 1] - off_h[p]);
            if ((int64_t)so[sl] + 32 * depth > 0x7fffffff)
                return fail(c, LSKUM_ERR_ARG, "too many stencil entries for the mixed layout");
            so[sl + 1] = so[sl] + 32 * depth;
        }
        const int64_t nslot = std::max<int32_t>(so[nslices], 1);
        CK(c, dalloc(c, &c->slice_off, nslices + 1));
        CK(c, cudaMemcpyAsync(c->slice_off, so.data(), (nslices + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        CK(c, dalloc(c, &c->s_idx, nslot));
        CK(c, dalloc(c, &c->s_ga, nslot));
        CK(c, dalloc(c, &c->s_gf, nslot));
        CK(c, dalloc(c, &c->s_fxw64, nslot));
        LAUNCH(c, launch_sell_fill(n, c->off, c->slice_off, c->idx, c->mask, dxy, lsw, fxw, c->fxw, c->mgeom(), s));
        CK(c, cudaFreeAsync(dxy, s));
        CK(c, cudaFreeAsync(lsw, s));
        CK(c, cudaFreeAsync(fxw, s));
        lskum_status st = build_tiles(c, off_h, so);
        if (st != LSKUM_OK) return st;
        CK(c, cudaStreamSynchronize(s));
    }
    CK(c, dalloc(c, &c->dt, n));
    CK(c, dalloc(c, &c->Rt, 4 * n));
    CK(c, dalloc(c, &c->Ut, 4 * n));
    CK(c, dalloc(c, &c->Ucm, 4 * n));
    CK(c, dalloc(c, &c->norm_part, residue_parts(n)));
    for (int k = 0; k < c->ncases; ++k)
        c->maxchunks = std::max(c->maxchunks, residue_chunks(c->case_start_h[k + 1] - c->case_start_h[k]));
    CK(c, dalloc(c, &c->norm_chunk, (int64_t)c->ncases * c->maxchunks));
    CK(c, dalloc(c, &c->status, 2));
    c->res_cap = 1024;
    CK(c, dalloc(c, &c->res_dev, (int64_t)c->res_cap * c->ncases));
    CK(c, dalloc(c, &c->res_counter, 1));
    CK(c, cudaMemsetAsync(c->res_counter, 0, sizeof(int), s));
    CK(c, cudaMemsetAsync(c->qgA, 0, 2 * 8 * n * qbytes, s));
    const int st_init[2] = {0, 0x7fffffff};
    CK(c, cudaMemcpyAsync(c->status, st_init, sizeof st_init, cudaMemcpyHostToDevice, s));
    if (c->kinetic) {
        // each case's free-stream q by the same kernel that turns states into q
        const double *uinf = c->case_uinf;
        if (!uinf) {
            double *u1 = nullptr;
            CK(c, dalloc(c, &u1, 4));
            CK(c, cudaMemcpyAsync(u1, c->gas.Uinf, 4 * sizeof(double), cudaMemcpyHostToDevice, s));
            uinf = u1;
        }
        if (c->mixed) {
            CK(c, dalloc(c, &c->qinf_f, 4 * c->ncases));
            LAUNCH(c, launch_q_from_U_mixed(c->ncases, c->gas, uinf, c->qinf_f, c->status, s));
        } else {
            CK(c, dalloc(c, &c->qinf, 4 * c->ncases));
            LAUNCH(c, launch_q_from_U(c->ncases, c->gas, uinf, c->qinf, c->status, s));
        }
    }
    if (c->ncases > 1) LAUNCH(c, launch_fill_state_cases(n, c->pcase, c->case_uinf, c->U, s));
    else LAUNCH(c, launch_fill_state(n, c->gas.Uinf, c->U, s));
    lskum_status st = refresh_q(c, c->U, c->q_cur);
    if (st != LSKUM_OK) return st;
    CK(c, cudaStreamSynchronize(s));
    return LSKUM_OK;
}

static lskum_status check_config(const lskum_config *cfg, int64_t n)
{
    if (cfg->order != 1 && cfg->order != 2) return fail(nullptr, LSKUM_ERR_ARG, "order must be 1 or 2");
    if (cfg->inner_iters < 0 || cfg->inner_iters > 1000) return fail(nullptr, LSKUM_ERR_ARG, "inner_iters out of range");
    if (cfg->time_scheme != 0 && cfg->time_scheme != 1) return fail(nullptr, LSKUM_ERR_ARG, "time_scheme must be 0 or 1");
    if (!(cfg->cfl > 0.0) || !(cfg->gamma > 1.0) || !(cfg->mach >= 0.0) || !std::isfinite(cfg->aoa_deg))
        return fail(nullptr, LSKUM_ERR_ARG, "cfl, gamma, mach or aoa out of range");
    if (cfg->precision != 0 && cfg->precision != 1)
        return fail(nullptr, LSKUM_ERR_ARG, "precision must be 0 (FP64) or 1 (mixed)");
    if (cfg->precision == 1 && n >= (int64_t)1 << 28)
        return fail(nullptr, LSKUM_ERR_ARG, "the mixed form takes at most 2^28 - 1 points");
    if (cfg->reorder < 0 || cfg->reorder > 2) return fail(nullptr, LSKUM_ERR_ARG, "reorder must be 0, 1 or 2");
    if (!(cfg->limiter_K >= 0.0) || !std::isfinite(cfg->limiter_K))
        return fail(nullptr, LSKUM_ERR_ARG, "limiter_K must be finite and >= 0");
    if (cfg->boundary != LSKUM_BOUNDARY_PLAIN && cfg->boundary != LSKUM_BOUNDARY_KINETIC)
        return fail(nullptr, LSKUM_ERR_ARG, "boundary must be 0 (plain) or 1 (kinetic)");
    return LSKUM_OK;
}

static lskum_status check_points(int64_t n, const double *x, const double *y, const double *nx, const double *ny,
                                 const int32_t *flags)
{
    for (int64_t p = 0; p < n; ++p) {
        if (flags[p] < 0 || flags[p] > 2) return fail(nullptr, LSKUM_ERR_ARG, "point %lld has flag %d", (long long)p, flags[p]);
        if (!std::isfinite(x[p]) || !std::isfinite(y[p]) || !std::isfinite(nx[p]) || !std::isfinite(ny[p]))
            return fail(nullptr, LSKUM_ERR_ARG, "point %lld has a non-finite coordinate or normal", (long long)p);
        const double nn = nx[p] * nx[p] + ny[p] * ny[p];
        if (fabs(nn - 1.0) > 1e-8) return fail(nullptr, LSKUM_ERR_ARG, "point %lld has a normal that is not unit", (long long)p);
    }
    return LSKUM_OK;
}

extern "C" lskum_status lskum_create(int64_t n, const double *x, const double *y, const double *nx,
                                     const double *ny, const int32_t *flags, const int32_t *nbr_offsets,
                                     const int32_t *nbr_idx, int64_t n_wall, const int32_t *wall_order,
                                     const lskum_config *cfg, void *cuda_stream, lskum_ctx **out)
{
    if (!out) return fail(nullptr, LSKUM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || n >= (int64_t)0x7fffffff) return fail(nullptr, LSKUM_ERR_ARG, "n = %lld out of range", (long long)n);
    if (!x || !y || !nx || !ny || !flags || !nbr_offsets || !nbr_idx || !cfg)
        return fail(nullptr, LSKUM_ERR_ARG, "a required input pointer is NULL");
    if (n_wall < 0 || n_wall > n || (n_wall > 0 && !wall_order))
        return fail(nullptr, LSKUM_ERR_ARG, "bad wall contour (n_wall = %lld)", (long long)n_wall);
    lskum_status cst = check_config(cfg, n);
    if (cst != LSKUM_OK) return cst;
    if ((cst = check_points(n, x, y, nx, ny, flags)) != LSKUM_OK) return cst;
    std::string msg;
    lskum_status st = validate_csr(n, nbr_offsets, nbr_idx, msg);
    if (st != LSKUM_OK) return fail(nullptr, st, "%s", msg.c_str());
    for (int64_t w = 0; w < n_wall; ++w)
        if (wall_order[w] < 0 || wall_order[w] >= n)
            return fail(nullptr, LSKUM_ERR_ARG, "wall_order[%lld] out of range", (long long)w);

    lskum_ctx *c = new lskum_ctx();
    c->n = n;
    c->nnz = nbr_offsets[n];
    c->n_wall = n_wall;
    c->cfg = *cfg;
    c->mixed = cfg->precision == 1;
    c->kinetic = cfg->boundary == LSKUM_BOUNDARY_KINETIC;
    c->stream = (cudaStream_t)cuda_stream;
    c->gas.gamma = cfg->gamma;
    c->gas.inv_gm1 = 1.0 / (cfg->gamma - 1.0);
    c->gas.hc = 0.5 * (c->gas.inv_gm1 + 1.0);
    c->gas.g14 = cfg->gamma == 1.4;
    freestream(cfg->gamma, cfg->mach, cfg->aoa_deg, c->gas.Uinf);
    c->case_start_h = {0, n};
    c->case_wall_h = {0, n_wall};
    c->case_mach = {cfg->mach};
    c->case_aoa = {cfg->aoa_deg};
    st = create_impl(c, x, y, nx, ny, flags, nbr_offsets, nbr_idx, wall_order);
    if (st != LSKUM_OK) {
        g_create_error = c->err;
        lskum_destroy(c);
        return st;
    }
    *out = c;
    return LSKUM_OK;
}

extern "C" lskum_status lskum_create_batch(int n_cases, const lskum_case *cases, const lskum_config *cfg,
                                           void *cuda_stream, lskum_ctx **out)
{
    if (!out) return fail(nullptr, LSKUM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n_cases < 1 || n_cases > 65535 || !cases || !cfg)
        return fail(nullptr, LSKUM_ERR_ARG, "n_cases = %d out of range [1, 65535], or a NULL argument", n_cases);
    int64_t N = 0, NNZ = 0, NW = 0;
    for (int k = 0; k < n_cases; ++k) {
        const lskum_case &a = cases[k];
        if (a.n < 32) return fail(nullptr, LSKUM_ERR_ARG, "case %d: n = %lld (a case needs at least 32 points)", k,
                                  (long long)a.n);
        if (!a.x || !a.y || !a.nx || !a.ny || !a.flags || !a.nbr_offsets || !a.nbr_idx)
            return fail(nullptr, LSKUM_ERR_ARG, "case %d: a required input pointer is NULL", k);
        if (a.n_wall < 0 || a.n_wall > a.n || (a.n_wall > 0 && !a.wall_order))
            return fail(nullptr, LSKUM_ERR_ARG, "case %d: bad wall contour", k);
        if (!(a.mach > 0.0) || !std::isfinite(a.mach) || !std::isfinite(a.aoa_deg))
            return fail(nullptr, LSKUM_ERR_ARG, "case %d: mach must be > 0 and aoa finite", k);
        std::string msg;
        lskum_status st = validate_csr(a.n, a.nbr_offsets, a.nbr_idx, msg);
        if (st != LSKUM_OK) return fail(nullptr, st, "case %d: %s", k, msg.c_str());
        if ((st = check_points(a.n, a.x, a.y, a.nx, a.ny, a.flags)) != LSKUM_OK) {
            const std::string m2 = g_create_error;
            return fail(nullptr, st, "case %d: %s", k, m2.c_str());
        }
        for (int64_t w = 0; w < a.n_wall; ++w)
            if (a.wall_order[w] < 0 || a.wall_order[w] >= a.n)
                return fail(nullptr, LSKUM_ERR_ARG, "case %d: wall_order[%lld] out of range", k, (long long)w);
        N += a.n;
        NNZ += a.nbr_offsets[a.n];
        NW += a.n_wall;
    }
    if (N >= (int64_t)0x7fffffff || NNZ >= (int64_t)0x7fffffff)
        return fail(nullptr, LSKUM_ERR_ARG, "the batch has too many points or edges for 32-bit indices");
    // the disjoint union of the cases' clouds, in case order
    std::vector<double> x(N), y(N), nx(N), ny(N);
    std::vector<int32_t> flags(N), off(N + 1), idx(NNZ), wall(std::max<int64_t>(NW, 1));
    lskum_ctx *c = new lskum_ctx();
    c->ncases = n_cases;
    c->case_start_h.assign(n_cases + 1, 0);
    c->case_wall_h.assign(n_cases + 1, 0);
    c->case_of_input.resize(N);
    int64_t p0 = 0, e0 = 0, w0 = 0;
    off[0] = 0;
    for (int k = 0; k < n_cases; ++k) {
        const lskum_case &a = cases[k];
        for (int64_t p = 0; p < a.n; ++p) {
            x[p0 + p] = a.x[p]; y[p0 + p] = a.y[p]; nx[p0 + p] = a.nx[p]; ny[p0 + p] = a.ny[p];
            flags[p0 + p] = a.flags[p];
            off[p0 + p + 1] = (int32_t)(e0 + a.nbr_offsets[p + 1]);
            c->case_of_input[p0 + p] = (uint16_t)k;
        }
        const int64_t m = a.nbr_offsets[a.n];
        for (int64_t e = 0; e < m; ++e) idx[e0 + e] = (int32_t)(p0 + a.nbr_idx[e]);
        for (int64_t w = 0; w < a.n_wall; ++w) wall[w0 + w] = (int32_t)(p0 + a.wall_order[w]);
        p0 += a.n;
        e0 += m;
        w0 += a.n_wall;
        c->case_start_h[k + 1] = p0;
        c->case_wall_h[k + 1] = w0;
        c->case_mach.push_back(a.mach);
        c->case_aoa.push_back(a.aoa_deg);
    }
    c->n = N;
    c->nnz = NNZ;
    c->n_wall = NW;
    c->cfg = *cfg;
    c->cfg.mach = cases[0].mach;
    c->cfg.aoa_deg = cases[0].aoa_deg;
    c->mixed = cfg->precision == 1;
    c->kinetic = cfg->boundary == LSKUM_BOUNDARY_KINETIC;
    c->stream = (cudaStream_t)cuda_stream;
    c->gas.gamma = cfg->gamma;
    c->gas.inv_gm1 = 1.0 / (cfg->gamma - 1.0);
    c->gas.hc = 0.5 * (c->gas.inv_gm1 + 1.0);
    c->gas.g14 = cfg->gamma == 1.4;
    freestream(cfg->gamma, cases[0].mach, cases[0].aoa_deg, c->gas.Uinf);
    lskum_status st = check_config(cfg, N);
    if (st != LSKUM_OK) {
        delete c;
        return st;
    }
    st = create_impl(c, x.data(), y.data(), nx.data(), ny.data(), flags.data(), off.data(), idx.data(), wall.data());
    if (st != LSKUM_OK) {
        g_create_error = c->err;
        lskum_destroy(c);
        return st;
    }
    *out = c;
    return LSKUM_OK;
}

extern "C" int lskum_case_count(const lskum_ctx *c) { return c ? c->ncases : 0; }

extern "C" lskum_status lskum_case_range(const lskum_ctx *c, int k, int64_t *first, int64_t *count,
                                         int64_t *wall_first, int64_t *wall_count)
{
    if (!c || k < 0 || k >= c->ncases) return LSKUM_ERR_ARG;
    if (first) *first = c->case_start_h[k];
    if (count) *count = c->case_start_h[k + 1] - c->case_start_h[k];
    if (wall_first) *wall_first = c->case_wall_h[k];
    if (wall_count) *wall_count = c->case_wall_h[k + 1] - c->case_wall_h[k];
    return LSKUM_OK;
}

// q-derivatives of the state whose q-variables are in q (E15 with the
// configured inner iterations, limiter on the last pass); returns the buffer
// holding the result
static lskum_status gradients(lskum_ctx *c, const void *q, void **qg_out, int inner, double limK)
{
    void *src = c->qgA, *dst = c->qgB;
    if (c->mixed) {
        const MixedGeom g = c->mgeom();
        const float *qf = (const float *)q;
        if (inner == 0) {
            TIMED_LAUNCH(c, LSKUM_KERNEL_QGRAD, launch_qgrad_mixed(g, qf, nullptr, nullptr, (float *)src, nullptr, limK,
                                                                   c->stream, c->var_qgrad));
        } else {
            // as in the FP64 form: the first-order result stays in qgG1
            float *g1 = (float *)c->qgG1, *ext = limK > 0.0 ? (float *)c->qext : nullptr;
            TIMED_LAUNCH(c, LSKUM_KERNEL_QGRAD, launch_qgrad_mixed(g, qf, nullptr, nullptr, g1, ext, 0.0, c->stream,
                                                                   c->var_qgrad));
            const float *old = g1;
            for (int k = 0; k < inner; ++k) {
                TIMED_LAUNCH(c, LSKUM_KERNEL_QGRAD, launch_qgrad_mixed(g, qf, old, g1, (float *)src, ext,
                                                                       k == inner - 1 ? limK : 0.0, c->stream,
                                                                       c->var_qgrad));
                old = (const float *)src;
                std::swap(src, dst);
            }
            std::swap(src, dst);
        }
    } else {
        const DevGeom g = c->geom();
        const double *qd = (const double *)q;
        if (inner == 0) {
            TIMED_LAUNCH(c, LSKUM_KERNEL_QGRAD, launch_qgrad(g, qd, nullptr, nullptr, (double *)src, nullptr, limK,
                                                             c->stream));
        } else {
            // the first-order result stays in qgG1 for every inner pass, the
            // iterates alternate between qgA and qgB
            double *g1 = (double *)c->qgG1, *ext = limK > 0.0 ? (double *)c->qext : nullptr;
            TIMED_LAUNCH(c, LSKUM_KERNEL_QGRAD, launch_qgrad(g, qd, nullptr, nullptr, g1, ext, 0.0, c->stream));
            const double *old = g1;
            for (int k = 0; k < inner; ++k) {
                TIMED_LAUNCH(c, LSKUM_KERNEL_QGRAD, launch_qgrad(g, qd, old, g1, (double *)src, ext,
                                                                 k == inner - 1 ? limK : 0.0, c->stream));
                old = (const double *)src;
                std::swap(src, dst);
            }
            std::swap(src, dst);
        }
    }
    *qg_out = src;
    return LSKUM_OK;
}

static lskum_status gradients(lskum_ctx *c, const void *q, void **qg_out)
{
    return gradients(c, q, qg_out, c->cfg.inner_iters, c->cfg.order == 2 ? c->cfg.limiter_K : 0.0);
}

// one launch of the fused flux kernel in the context's precision
// (mode 0: residual into R; 1: forward Euler; 2: RK4 stage)
static lskum_status flux(lskum_ctx *c, const void *q, const void *qg, double *Uout, void *qout, int mode,
                         int stage, double *R)
{
    if (c->mixed) {
        MixedFluxParams P{};
        P.g = c->mgeom();
        P.nrm64 = c->nrm;
        P.q = (const float *)q;
        P.qg = (const float *)qg;
        P.Un = c->U;
        P.Uout = Uout;
        P.acc = c->acc;
        P.qout = (float *)qout;
        P.dt = c->dt;
        P.R = R;
        P.norm_part = c->norm_part;
        P.status = c->status;
        P.pcase = c->pcase;
        P.case_uinf = c->case_uinf;
        for (int k = 0; k < 4; ++k) P.Uinf[k] = c->gas.Uinf[k];
        P.gamma = (float)c->gas.gamma;
        P.inv_gm1 = (float)c->gas.inv_gm1;
        P.cfl = (float)c->cfg.cfl;
        P.g14 = c->gas.g14;
        P.order = c->cfg.order;
        P.mode = mode;
        P.stage = stage;
        TIMED_LAUNCH(c, LSKUM_KERNEL_FLUX, launch_flux_mixed(P, c->stream, c->var_flux));
    } else {
        FluxLaunch L{};
        L.q = (const double *)q;
        L.qg = (const double *)qg;
        L.Un = c->U;
        L.Uout = Uout;
        L.acc = c->acc;
        L.qout = (double *)qout;
        L.dt = c->dt;
        L.R = R;
        L.norm_part = c->norm_part;
        L.status = c->status;
        L.pcase = c->pcase;
        L.case_uinf = c->case_uinf;
        L.cfl = c->cfg.cfl;
        L.order = c->cfg.order;
        L.mode = mode;
        L.stage = stage;
        TIMED_LAUNCH(c, LSKUM_KERNEL_FLUX, launch_flux(c->geom(), c->gas, L, c->stream));
    }
    return LSKUM_OK;
}

static lskum_status iteration(lskum_ctx *c)
{
    const bool rk4 = c->cfg.time_scheme == 1;
    const int stages = rk4 ? 4 : 1;
    for (int k = 0; k < stages; ++k) {
        void *qg = nullptr;
        lskum_status st;
        if (c->cfg.order == 2 && (st = gradients(c, c->q_cur, &qg)) != LSKUM_OK) return st;
        st = flux(c, c->q_cur, qg, (rk4 && k < 3) ? c->Us : c->U, c->q_nxt, rk4 ? 2 : 1, k, nullptr);
        if (st != LSKUM_OK) return st;
        std::swap(c->q_cur, c->q_nxt);
        if (k == 0) c->launches++;  // the residue reduction is two kernels
        if (k == 0)
            LAUNCH(c, launch_residue_finish(c->norm_part, c->case_start, c->ncases, c->maxchunks, c->norm_chunk,
                                            c->res_dev, c->res_counter, c->res_cap, c->stream));
    }
    return LSKUM_OK;
}

static lskum_status reset_status(lskum_ctx *c)
{
    const int st_init[2] = {0, 0x7fffffff};
    CK(c, cudaMemcpyAsync(c->status, st_init, sizeof st_init, cudaMemcpyHostToDevice, c->stream));
    return LSKUM_OK;
}

static lskum_status read_status(lskum_ctx *c, int st[2])
{
    CK(c, cudaMemcpyAsync(st, c->status, 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return LSKUM_OK;
}

// captures `iters` iterations from the current q buffer into g (the kernels
// only: status, counter and backup are set up outside the graph)
static lskum_status capture_step_graph(lskum_ctx *c, lskum_ctx::StepGraph &g, int iters)
{
    if (!c->gstream) CK(c, cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking));
    if (g.exec) {
        CK(c, cudaGraphExecDestroy(g.exec));
        g.exec = nullptr;
    }
    void *const q_start = c->q_cur, *const q_other = c->q_nxt;
    cudaStream_t user = c->stream;
    const int64_t launches0 = c->launches;
    CK(c, cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal));
    c->stream = c->gstream;
    lskum_status st = LSKUM_OK;
    for (int i = 0; i < iters && st == LSKUM_OK; ++i) st = iteration(c);
    c->stream = user;
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(c->gstream, &graph);
    // the capture only recorded the launches: undo the q ping-pong (a replay
    // ends on q_start again) and the launch count
    c->q_cur = q_start;
    c->q_nxt = q_other;
    g.launches = c->launches - launches0;
    c->launches = launches0;
    if (st != LSKUM_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    CK(c, ec);
    const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(c, ei);
    g.q_start = q_start;
    g.res = c->res_dev;
    g.iters = iters;
    return LSKUM_OK;
}

// n_iters iterations by graph replay; returns the iterations left to launch
// directly (an odd forward-Euler remainder)
static lskum_status replay_step_graph(lskum_ctx *c, int n_iters, int *left)
{
    const int per = c->cfg.time_scheme == 1 ? 1 : 2;
    *left = n_iters % per;
    const int reps = n_iters / per;
    if (reps == 0) return LSKUM_OK;
    lskum_ctx::StepGraph *g = nullptr;
    for (auto &cand : c->graphs)
        if (cand.exec && cand.q_start == c->q_cur && cand.res == c->res_dev) g = &cand;
    if (!g) {
        g = &c->graphs[c->q_cur < c->q_nxt ? 0 : 1];  // one slot per q buffer
        lskum_status st = capture_step_graph(c, *g, per);
        if (st != LSKUM_OK) return st;
    }
    for (int r = 0; r < reps; ++r) {
        CK(c, cudaGraphLaunch(g->exec, c->stream));
        c->launches += g->launches;
    }
    return LSKUM_OK;
}

extern "C" lskum_status lskum_step(lskum_ctx *c, int n_iters, double *res_history)
{
    if (!c) return LSKUM_ERR_ARG;
    NvtxRange nvtx_("lskum_step");
    c->err.clear();
    if (n_iters < 0) return fail(c, LSKUM_ERR_ARG, "n_iters < 0");
    if (n_iters == 0) return LSKUM_OK;
    if (n_iters > c->res_cap) {
        double *r = nullptr;
        CK(c, dalloc(c, &r, (int64_t)n_iters * c->ncases));
        c->res_dev = r;
        c->res_cap = n_iters;
    }
    lskum_status st = reset_status(c);
    if (st != LSKUM_OK) return st;
    CK(c, cudaMemcpyAsync(c->Ubak, c->U, 4 * c->n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    CK(c, cudaMemsetAsync(c->res_counter, 0, sizeof(int), c->stream));
    int direct = n_iters;
    if (!c->profiling && !c->graphs_off) {
        st = replay_step_graph(c, n_iters, &direct);
        if (st != LSKUM_OK) return st;
    }
    for (int it = 0; it < direct; ++it) {
        st = iteration(c);
        if (st != LSKUM_OK) return st;
    }
    if (res_history)
        CK(c, cudaMemcpyAsync(res_history, c->res_dev, (size_t)n_iters * c->ncases * sizeof(double),
                              cudaMemcpyDeviceToHost, c->stream));
    int sh[2];
    st = read_status(c, sh);
    if (st != LSKUM_OK) return st;
    if (sh[0] & STATUS_NONPHYSICAL) {
        CK(c, cudaMemcpyAsync(c->U, c->Ubak, 4 * c->n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
        if ((st = refresh_q(c, c->U, c->q_cur)) != LSKUM_OK) return st;
        CK(c, cudaStreamSynchronize(c->stream));
        return fail(c, LSKUM_ERR_NONPHYSICAL,
                    "non-physical state (rho <= 0, p <= 0 or non-finite) at point %d; state rolled back",
                    c->perm_h[sh[1]]);
    }
    return LSKUM_OK;
}

// q-variables of a caller state (device [4][n], input order) into q_nxt, or the
// context's own q
static lskum_status q_of(lskum_ctx *c, const double *U, const void **q)
{
    if (!U) {
        *q = c->q_cur;
        return LSKUM_OK;
    }
    LAUNCH(c, launch_state_in(c->n, c->perm, U, c->Ut, c->stream));
    lskum_status st = refresh_q(c, c->Ut, c->q_nxt);
    if (st != LSKUM_OK) return st;
    *q = c->q_nxt;
    return LSKUM_OK;
}

static lskum_status check_nonphysical(lskum_ctx *c)
{
    int sh[2];
    lskum_status st = read_status(c, sh);
    if (st != LSKUM_OK) return st;
    if (sh[0] & STATUS_NONPHYSICAL)
        return fail(c, LSKUM_ERR_NONPHYSICAL, "non-physical state at point %d", c->perm_h[sh[1]]);
    return LSKUM_OK;
}

extern "C" lskum_status lskum_residual(lskum_ctx *c, const double *U, double *R)
{
    if (!c) return LSKUM_ERR_ARG;
    NvtxRange nvtx_("lskum_residual");
    c->err.clear();
    if (!R) return fail(c, LSKUM_ERR_ARG, "R is NULL");
    lskum_status st = reset_status(c);
    if (st != LSKUM_OK) return st;
    const void *q = nullptr;
    if ((st = q_of(c, U, &q)) != LSKUM_OK) return st;
    void *qg = nullptr;
    if (c->cfg.order == 2 && (st = gradients(c, q, &qg)) != LSKUM_OK) return st;
    if ((st = flux(c, q, qg, nullptr, nullptr, 0, 0, c->Rt)) != LSKUM_OK) return st;
    LAUNCH(c, launch_state_out(c->n, c->perm, c->Rt, R, c->stream));
    return check_nonphysical(c);
}

// second order with the limiter on
static bool limited(const lskum_ctx *c) { return c->cfg.order == 2 && c->cfg.limiter_K > 0.0; }

// the final q-derivative iterate of the FP64 forward recomputation (vjp_forward)
static const double *vjp_final_gradient(const lskum_ctx *c)
{
    if (c->cfg.order != 2) return nullptr;
    return limited(c) ? c->vGlim : c->vG + (int64_t)c->cfg.inner_iters * 8 * c->n;
}

static lskum_status vjp_workspace(lskum_ctx *c)
{
    if (c->vjp_ready) return LSKUM_OK;
    const int64_t n = c->n, m = std::max<int64_t>(c->nnz, 1);
    const int K = c->cfg.order == 2 ? c->cfg.inner_iters : 0;
    CK(c, dalloc(c, &c->vq, 4 * n));
    if (c->cfg.order == 2) {
        CK(c, dalloc(c, &c->vG, (int64_t)(K + 1) * 8 * n));
        CK(c, dalloc(c, &c->vgb, 8 * n));
        CK(c, dalloc(c, &c->vgb2, 8 * n));
    }
    CK(c, dalloc(c, &c->vRb, 4 * n));
    CK(c, dalloc(c, &c->vqb, 4 * n));
    CK(c, dalloc(c, &c->vebar, 4 * m));
    CK(c, dalloc(c, &c->vwbar, m));
    CK(c, dalloc(c, &c->vabar, m));
    CK(c, dalloc(c, &c->vdbar, m));
    CK(c, dalloc(c, &c->toff, n + 1));
    CK(c, dalloc(c, &c->tedge, m));
    CK(c, dalloc(c, &c->tsrc, m));
    CK(c, dalloc(c, &c->vUacc, 4 * n));
    CK(c, dalloc(c, &c->vpxy, n));
    CK(c, dalloc(c, &c->fdsb, std::max<int64_t>(c->n_wall, 1)));
    if (limited(c)) {
        CK(c, dalloc(c, &c->vGlim, 8 * n));
        CK(c, dalloc(c, &c->vext, 4 * n));
        CK(c, dalloc(c, &c->vlidx, 4 * n));
        CK(c, dalloc(c, &c->vlval, 4 * n));
    }
    c->launches += 4;
    LAUNCH(c, build_transpose_csr(n, c->nnz, c->off, c->idx, c->toff, c->tedge, c->tsrc, c->stream));
    c->vjp_ready = true;
    return LSKUM_OK;
}

static AdjParams adj_params(lskum_ctx *c)
{
    const int64_t n = c->n;
    const int K = c->cfg.order == 2 ? c->cfg.inner_iters : 0;
    AdjParams P{};
    P.g = c->geom();
    P.q = c->vq;
    P.qg = vjp_final_gradient(c);
    P.Rbar = c->vRb;
    P.qbar = c->vqb;
    P.gbar = c->vgb;
    P.ebar = c->vebar;
    P.wbar = c->vwbar;
    P.abar = c->vabar;
    P.dbar = c->vdbar;
    P.toff = c->toff;
    P.tedge = c->tedge;
    P.tsrc = c->tsrc;
    P.perm = c->perm;
    P.inv_gm1 = c->gas.inv_gm1;
    P.g14 = c->gas.g14;
    P.order = c->cfg.order;
    return P;
}

// FP64 q and q-derivative iterates of an internal state (vq, vG; with the
// limiter also the limited last iterate vGlim, the forward's last pass run
// again with the limiter)
static lskum_status vjp_forward(lskum_ctx *c, const double *Ui)
{
    const int64_t n = c->n;
    const int K = c->cfg.inner_iters;
    const DevGeom g = c->geom();
    LAUNCH(c, launch_q_from_U(n, c->gas, Ui, c->vq, c->status, c->stream));
    if (c->cfg.order == 2) {
        const double limK = c->cfg.limiter_K;
        double *ext = limited(c) && K > 0 ? c->vext : nullptr;
        LAUNCH(c, launch_qgrad(g, c->vq, nullptr, nullptr, c->vG, ext, 0.0, c->stream));
        for (int k = 1; k <= K; ++k)
            LAUNCH(c, launch_qgrad(g, c->vq, c->vG + (int64_t)(k - 1) * 8 * n, c->vG, c->vG + (int64_t)k * 8 * n,
                                   nullptr, 0.0, c->stream));
        if (limited(c)) {
            if (K == 0) LAUNCH(c, launch_qgrad(g, c->vq, nullptr, nullptr, c->vGlim, nullptr, limK, c->stream));
            else
                LAUNCH(c, launch_qgrad(g, c->vq, c->vG + (int64_t)(K - 1) * 8 * n, c->vG, c->vGlim, ext, limK,
                                       c->stream));
        }
    }
    return LSKUM_OK;
}

// FP64 residual of an internal state (Rout internal [n][4]); leaves vq, vG at that state
static lskum_status residual_fp64(lskum_ctx *c, const double *Ui, double *Rout)
{
    lskum_status st = vjp_forward(c, Ui);
    if (st != LSKUM_OK) return st;
    FluxLaunch L{};
    L.q = c->vq;
    L.qg = vjp_final_gradient(c);
    L.R = Rout;
    L.norm_part = c->norm_part;
    L.status = c->status;
    L.pcase = c->pcase;
    L.case_uinf = c->case_uinf;
    L.cfl = c->cfg.cfl;
    L.order = c->cfg.order;
    L.mode = 0;
    LAUNCH(c, launch_flux(c->geom(), c->gas, L, c->stream));
    return LSKUM_OK;
}

// FP32 workspace of the residual VJP
static lskum_status fvjp_workspace(lskum_ctx *c)
{
    if (c->fvjp_ready) return LSKUM_OK;
    const int64_t n = c->n, m = std::max<int64_t>(c->nnz, 1);
    const int K = c->cfg.order == 2 ? c->cfg.inner_iters : 0;
    CK(c, dalloc(c, &c->fq, 4 * n));
    if (c->cfg.order == 2) {
        CK(c, dalloc(c, &c->fG, (int64_t)(K + 1) * 8 * n));
        CK(c, dalloc(c, &c->fgb, 8 * n));
        CK(c, dalloc(c, &c->fgb2, 8 * n));
    }
    CK(c, dalloc(c, &c->fRb, 4 * n));
    CK(c, dalloc(c, &c->fqb, 4 * n));
    CK(c, dalloc(c, &c->febar, 4 * m));
    c->fvjp_ready = true;
    return LSKUM_OK;
}

// the FP32 product: the mixed form's FP32 q and q-derivative passes forward,
// the reverse pass in FP32, the geometry cotangents and E13 Jacobian in FP64
static lskum_status vjp_residual_fp32(lskum_ctx *c, const double *Ui, double *Ub_acc, bool geom)
{
    const int64_t n = c->n;
    const bool second = c->cfg.order == 2;
    const int K = second ? c->cfg.inner_iters : 0;
    lskum_status st = fvjp_workspace(c);
    if (st != LSKUM_OK) return st;
    const MixedGeom mg = c->mgeom();
    LAUNCH(c, launch_q_from_U_mixed(n, c->gas, Ui, c->fq, c->status, c->stream));
    if (second) {
        LAUNCH(c, launch_qgrad_mixed(mg, c->fq, nullptr, nullptr, c->fG, nullptr, 0.0, c->stream, c->var_qgrad));
        for (int k = 1; k <= K; ++k)
            LAUNCH(c, launch_qgrad_mixed(mg, c->fq, c->fG + (int64_t)(k - 1) * 8 * n, c->fG,
                                         c->fG + (int64_t)k * 8 * n, nullptr, 0.0, c->stream, c->var_qgrad));
    }
    LAUNCH(c, launch_to_float(4 * n, c->vRb, c->fRb, c->stream));
    const AdjParams Pd = adj_params(c);
    AdjParamsT<float> P{};
    P.g = Pd.g;
    P.q = c->fq;
    P.qg = second ? c->fG + (int64_t)K * 8 * n : nullptr;
    P.Rbar = c->fRb;
    P.qbar = c->fqb;
    P.gbar = c->fgb;
    P.ebar = c->febar;
    P.wbar = Pd.wbar;
    P.abar = Pd.abar;
    P.dbar = Pd.dbar;
    P.toff = Pd.toff;
    P.tedge = Pd.tedge;
    P.tsrc = Pd.tsrc;
    P.perm = Pd.perm;
    P.inv_gm1 = Pd.inv_gm1;
    P.g14 = Pd.g14;
    P.order = Pd.order;
    c->launches++;
    LAUNCH(c, launch_adj_flux(P, c->stream));
    if (second) {
        CK(c, cudaMemsetAsync(c->vabar, 0, std::max<int64_t>(c->nnz, 1) * sizeof(double2), c->stream));
        float *gin = c->fgb, *gout = c->fgb2;
        for (int k = K; k >= 1; --k) {
            LAUNCH(c, launch_adj_grad(P, (const float *)(c->fG + (int64_t)(k - 1) * 8 * n), (const float *)gin,
                                      gout, c->stream));
            std::swap(gin, gout);
        }
        LAUNCH(c, launch_adj_grad(P, (const float *)nullptr, (const float *)gin, (float *)nullptr, c->stream));
    }
    if (geom) LAUNCH(c, launch_adj_weights(Pd, c->stream));
    LAUNCH(c, launch_adj_state(P, Ui, Ub_acc, c->stream));
    return LSKUM_OK;
}

// one residual VJP at the internal state Ui for the internal cotangent vRb:
// Ub_acc ([n][4], internal) += (dR/dU)^T R_bar; vdbar += the offset
// cotangents (the caller zeroes vdbar once per product)
static lskum_status vjp_residual(lskum_ctx *c, const double *Ui, double *Ub_acc, bool geom, bool fwd_done)
{
    const int64_t n = c->n;
    const bool second = c->cfg.order == 2;
    const int K = second ? c->cfg.inner_iters : 0;
    lskum_status st;
    if (!fwd_done && (st = vjp_forward(c, Ui)) != LSKUM_OK) return st;
    const AdjParams P = adj_params(c);
    c->launches++;
    LAUNCH(c, launch_adj_flux(P, c->stream));
    if (second) {
        CK(c, cudaMemsetAsync(c->vabar, 0, std::max<int64_t>(c->nnz, 1) * sizeof(double2), c->stream));
        double *gin = c->vgb, *gout = c->vgb2;
        if (limited(c)) {
            // the limiter first: the flux saw the limited last iterate
            c->launches++;
            LAUNCH(c, launch_adj_limit(P, c->vG + (int64_t)K * 8 * n, gin, gout, c->vlidx, c->vlval,
                                       c->cfg.limiter_K, c->stream));
            std::swap(gin, gout);
        }
        for (int k = K; k >= 1; --k) {
            LAUNCH(c, launch_adj_grad(P, c->vG + (int64_t)(k - 1) * 8 * n, gin, gout, c->stream));
            std::swap(gin, gout);
        }
        LAUNCH(c, launch_adj_grad(P, (const double *)nullptr, (const double *)gin, (double *)nullptr, c->stream));
    }
    if (geom) LAUNCH(c, launch_adj_weights(P, c->stream));
    LAUNCH(c, launch_adj_state(P, Ui, Ub_acc, c->stream));
    return LSKUM_OK;
}

static lskum_status vjp_begin(lskum_ctx *c)
{
    if (c->kinetic)
        return fail(c, LSKUM_ERR_ARG, "derivatives need boundary = 0 (the mirror images are not differentiated)");
    lskum_status st = vjp_workspace(c);
    if (st != LSKUM_OK) return st;
    if ((st = reset_status(c)) != LSKUM_OK) return st;
    CK(c, cudaMemsetAsync(c->vdbar, 0, std::max<int64_t>(c->nnz, 1) * sizeof(double2), c->stream));
    CK(c, cudaMemsetAsync(c->vpxy, 0, c->n * sizeof(double2), c->stream));
    CK(c, cudaMemsetAsync(c->vUacc, 0, 4 * c->n * sizeof(double), c->stream));
    return LSKUM_OK;
}

// outputs of a product: U_bar from vUacc, x_bar / y_bar from vdbar and vpxy (input order)
static lskum_status vjp_end(lskum_ctx *c, double *U_bar, double *x_bar, double *y_bar, int flags)
{
    if (flags & ~LSKUM_VJP_ACCUMULATE_XY) return fail(c, LSKUM_ERR_ARG, "unknown flags 0x%x", flags);
    if (x_bar || y_bar)
        LAUNCH(c, launch_adj_points(adj_params(c), c->vpxy, x_bar, y_bar, (flags & LSKUM_VJP_ACCUMULATE_XY) != 0,
                                    c->stream));
    if (U_bar) LAUNCH(c, launch_state_out(c->n, c->perm, c->vUacc, U_bar, c->stream));
    return check_nonphysical(c);
}

extern "C" lskum_status lskum_residual_vjp(lskum_ctx *c, const double *U, const double *R_bar, double *U_bar,
                                           double *x_bar, double *y_bar, int flags)
{
    if (!c) return LSKUM_ERR_ARG;
    NvtxRange nvtx_("lskum_residual_vjp");
    c->err.clear();
    if (!R_bar) return fail(c, LSKUM_ERR_ARG, "R_bar is NULL");
    if (!U_bar && !x_bar && !y_bar) return LSKUM_OK;
    lskum_status st = vjp_begin(c);
    if (st != LSKUM_OK) return st;
    const double *Ui = c->U;
    if (U) {
        LAUNCH(c, launch_state_in(c->n, c->perm, U, c->Ut, c->stream));
        Ui = c->Ut;
    }
    LAUNCH(c, launch_state_in(c->n, c->perm, R_bar, c->vRb, c->stream));
    if (flags & LSKUM_VJP_FP32) {
        if (!c->mixed) return fail(c, LSKUM_ERR_ARG, "the FP32 product needs a mixed-precision context");
        if (limited(c))
            return fail(c, LSKUM_ERR_ARG, "the FP32 product needs limiter_K = 0 (the FP64 product covers the limiter)");
        if ((st = vjp_residual_fp32(c, Ui, c->vUacc, x_bar || y_bar)) != LSKUM_OK) return st;
    } else if ((st = vjp_residual(c, Ui, c->vUacc, x_bar || y_bar, false)) != LSKUM_OK) {
        return st;
    }
    return vjp_end(c, U_bar, x_bar, y_bar, flags & ~LSKUM_VJP_FP32);
}

static lskum_status step_vjp_workspace(lskum_ctx *c)
{
    if (c->svjp_ready) return LSKUM_OK;
    const int64_t n = c->n;
    for (auto &b : c->sR) CK(c, dalloc(c, &b, 4 * n));
    for (auto &b : c->sRb) CK(c, dalloc(c, &b, 4 * n));
    for (auto &b : c->sU) CK(c, dalloc(c, &b, 4 * n));
    CK(c, dalloc(c, &c->sUb, 4 * n));
    CK(c, dalloc(c, &c->sUin, 4 * n));
    CK(c, dalloc(c, &c->sdt, n));
    CK(c, dalloc(c, &c->sdtb, n));
    c->svjp_ready = true;
    return LSKUM_OK;
}

extern "C" lskum_status lskum_step_vjp(lskum_ctx *c, const double *U, const double *U_bar_next, double *U_bar,
                                       double *x_bar, double *y_bar, int flags)
{
    if (!c) return LSKUM_ERR_ARG;
    NvtxRange nvtx_("lskum_step_vjp");
    c->err.clear();
    if (!U_bar_next) return fail(c, LSKUM_ERR_ARG, "U_bar_next is NULL");
    if (!U_bar && !x_bar && !y_bar) return LSKUM_OK;
    lskum_status st = vjp_begin(c);
    if (st != LSKUM_OK) return st;
    if ((st = step_vjp_workspace(c)) != LSKUM_OK) return st;
    const int64_t n = c->n;
    const bool geom = x_bar || y_bar;
    const double *Un = c->U;
    if (U) {
        LAUNCH(c, launch_state_in(n, c->perm, U, c->sUin, c->stream));
        Un = c->sUin;
    }
    LAUNCH(c, launch_state_in(n, c->perm, U_bar_next, c->sUb, c->stream));
    StageParams S{};
    S.n = n;
    S.flag = c->flag;
    S.nrm = c->nrm;
    S.dt = c->sdt;
    S.pcase = c->pcase;
    S.case_uinf = c->case_uinf;
    for (int k = 0; k < 4; ++k) S.Uinf[k] = c->gas.Uinf[k];
    // forward: dt frozen at U^n, the stage states and residuals (FP64)
    LAUNCH(c, launch_timestep(n, c->gas, c->cfg.cfl, c->dmin, Un, c->sdt, c->stream));
    if ((st = residual_fp64(c, Un, c->sR[0])) != LSKUM_OK) return st;
    if (c->cfg.time_scheme == 0) {
        // U^{n+1} = P(U^n - dt R(U^n))
        LAUNCH(c, launch_stage_adj(S, c->sUb, c->sR[0], 1.0, true, c->vUacc, c->sdtb, c->vRb, c->stream));
        if ((st = vjp_residual(c, Un, c->vUacc, geom, true)) != LSKUM_OK) return st;
    } else {
        // U_{k+1} = P(U^n - c_k dt R_k), R_{k+1} = R(U_{k+1}); U_{k+1} is kept in sU[k]
        const double cst[3] = {0.5, 0.5, 1.0};
        for (int k = 0; k < 3; ++k) {
            LAUNCH(c, launch_stage_fwd(S, Un, c->sR[k], cst[k], c->sU[k], c->stream));
            if ((st = residual_fp64(c, c->sU[k], c->sR[k + 1])) != LSKUM_OK) return st;
        }
        // reverse: the last stage, then stages 2, 1, 0 (their residuals R3, R2, R1, R0)
        const double *Rs[4] = {c->sR[0], c->sR[1], c->sR[2], c->sR[3]};
        LAUNCH(c, launch_stage_adj_rk4_final(S, c->sUb, Rs, c->vUacc, c->sdtb, c->sRb, c->stream));
        for (int k = 3; k >= 1; --k) {
            // the cotangent of the stage state U_k from R_k = R(U_k)
            CK(c, cudaMemsetAsync(c->sUb, 0, 4 * n * sizeof(double), c->stream));
            CK(c, cudaMemcpyAsync(c->vRb, c->sRb[k], 4 * n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
            if ((st = vjp_residual(c, c->sU[k - 1], c->sUb, geom, false)) != LSKUM_OK) return st;
            // U_k = P(U^n - c_k dt R_{k-1})
            LAUNCH(c, launch_stage_adj(S, c->sUb, c->sR[k - 1], cst[k - 1], false, c->vUacc, c->sdtb,
                                       c->sRb[k - 1], c->stream));
        }
        CK(c, cudaMemcpyAsync(c->vRb, c->sRb[0], 4 * n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
        if ((st = vjp_residual(c, Un, c->vUacc, geom, false)) != LSKUM_OK) return st;
    }
    LAUNCH(c, launch_dt_adj(S, c->geom(), c->cfg.cfl, c->gas.inv_gm1, Un, c->sdtb, c->vUacc, c->vdbar, c->stream));
    return vjp_end(c, U_bar, x_bar, y_bar, flags);
}

extern "C" lskum_status lskum_forces_vjp(lskum_ctx *c, int k, double cl_bar, double cd_bar, double *U_bar,
                                         double *x_bar, double *y_bar, int flags)
{
    if (!c) return LSKUM_ERR_ARG;
    NvtxRange nvtx_("lskum_forces_vjp");
    c->err.clear();
    if (k < 0 || k >= c->ncases) return fail(c, LSKUM_ERR_ARG, "case %d out of range", k);
    const int64_t w0 = c->case_wall_h[k], nw = c->case_wall_h[k + 1] - w0;
    if (nw == 0) return fail(c, LSKUM_ERR_ARG, "no wall contour was given at create for case %d", k);
    const double qinf = 0.5 * c->case_mach[k] * c->case_mach[k];
    if (!(qinf > 0.0)) return fail(c, LSKUM_ERR_ARG, "forces need mach > 0");
    if (!U_bar && !x_bar && !y_bar) return LSKUM_OK;
    lskum_status st = vjp_workspace(c);
    if (st != LSKUM_OK) return st;
    if ((st = reset_status(c)) != LSKUM_OK) return st;
    CK(c, cudaMemsetAsync(c->vdbar, 0, std::max<int64_t>(c->nnz, 1) * sizeof(double2), c->stream));
    CK(c, cudaMemsetAsync(c->vpxy, 0, c->n * sizeof(double2), c->stream));
    CK(c, cudaMemsetAsync(c->vUacc, 0, 4 * c->n * sizeof(double), c->stream));
    const double a = c->case_aoa[k] * 3.14159265358979323846 / 180.0;
    // Cl = fy cos a - fx sin a, Cd = fx cos a + fy sin a
    const double fxb = -cl_bar * sin(a) + cd_bar * cos(a), fyb = cl_bar * cos(a) + cd_bar * sin(a);
    c->launches++;
    LAUNCH(c, launch_forces_adj(nw, c->gas.gamma, qinf, c->wall + w0, c->wall_ds + w0, c->nrm, c->xy, c->U, fxb,
                                fyb, c->vUacc, c->fdsb + w0, c->vpxy, c->stream));
    return vjp_end(c, U_bar, x_bar, y_bar, flags);
}

extern "C" lskum_status lskum_q_derivatives(lskum_ctx *c, const double *U, double *qx, double *qy)
{
    if (!c) return LSKUM_ERR_ARG;
    NvtxRange nvtx_("lskum_q_derivatives");
    c->err.clear();
    if (!qx || !qy) return fail(c, LSKUM_ERR_ARG, "qx or qy is NULL");
    lskum_status st = reset_status(c);
    if (st != LSKUM_OK) return st;
    const void *q = nullptr;
    if ((st = q_of(c, U, &q)) != LSKUM_OK) return st;
    void *qg = nullptr;
    const bool second = c->cfg.order == 2;
    st = gradients(c, q, &qg, second ? c->cfg.inner_iters : 0, second ? c->cfg.limiter_K : 0.0);
    if (st != LSKUM_OK) return st;
    if (c->mixed) LAUNCH(c, launch_grad_out_f(c->n, c->perm, (const float *)qg, qx, qy, c->stream));
    else LAUNCH(c, launch_grad_out(c->n, c->perm, (const double *)qg, qx, qy, c->stream));
    return check_nonphysical(c);
}

extern "C" lskum_status lskum_timestep(lskum_ctx *c, const double *U, double *dt)
{
    if (!c) return LSKUM_ERR_ARG;
    c->err.clear();
    if (!dt) return fail(c, LSKUM_ERR_ARG, "dt is NULL");
    const double *Ui = c->U;
    if (U) {
        LAUNCH(c, launch_state_in(c->n, c->perm, U, c->Ut, c->stream));
        Ui = c->Ut;
    }
    LAUNCH(c, launch_timestep(c->n, c->gas, c->cfg.cfl, c->dmin, Ui, c->Rt, c->stream));
    LAUNCH(c, launch_scalar_out(c->n, c->perm, c->Rt, dt, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return LSKUM_OK;
}

static void drop_graphs(lskum_ctx *c)
{
    for (auto &g : c->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g = lskum_ctx::StepGraph{};
    }
}

extern "C" lskum_status lskum_set_tuning(lskum_ctx *c, int flux_variant, int qgrad_variant)
{
    if (!c) return LSKUM_ERR_ARG;
    c->err.clear();
    if (!c->mixed) return fail(c, LSKUM_ERR_ARG, "launch-shape variants exist for the mixed-precision kernels only");
    if (flux_variant < 0 || flux_variant >= mixed_variants(0) || qgrad_variant < 0 ||
        qgrad_variant >= mixed_variants(1))
        return fail(c, LSKUM_ERR_ARG, "variant out of range");
    CK(c, cudaStreamSynchronize(c->stream));
    c->var_flux = flux_variant;
    c->var_qgrad = qgrad_variant;
    drop_graphs(c);
    return LSKUM_OK;
}

extern "C" lskum_status lskum_mixed_fp64_points(lskum_ctx *c, int64_t *count)
{
    if (!c || !count) return LSKUM_ERR_ARG;
    c->err.clear();
    *count = c->mixed ? (int64_t)c->n_fp64_closure : 0;
    return LSKUM_OK;
}

// times `reps` launches of one variant on the context's stream (milliseconds per launch)
template <class F>
static lskum_status time_variant(lskum_ctx *c, int reps, cudaEvent_t e0, cudaEvent_t e1, F launch, double *ms)
{
    CK(c, launch());  // warm-up
    CK(c, cudaEventRecord(e0, c->stream));
    for (int r = 0; r < reps; ++r) CK(c, launch());
    CK(c, cudaEventRecord(e1, c->stream));
    CK(c, cudaEventSynchronize(e1));
    float t = 0.0f;
    CK(c, cudaEventElapsedTime(&t, e0, e1));
    c->launches += reps + 1;
    *ms = (double)t / reps;
    return LSKUM_OK;
}

extern "C" lskum_status lskum_autotune(lskum_ctx *c, int reps, lskum_tuning *out)
{
    if (!c) return LSKUM_ERR_ARG;
    NvtxRange nvtx_("lskum_autotune");
    c->err.clear();
    if (!c->mixed) return fail(c, LSKUM_ERR_ARG, "the autotuner covers the mixed-precision kernels (precision = 1)");
    if (reps < 1) reps = 5;
    lskum_status st = reset_status(c);
    if (st != LSKUM_OK) return st;
    CK(c, cudaStreamSynchronize(c->stream));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(c, cudaEventCreate(&e0));
    cudaError_t ee = cudaEventCreate(&e1);
    if (ee != cudaSuccess) {
        cudaEventDestroy(e0);
        CK(c, ee);
    }
    const MixedGeom g = c->mgeom();
    const float *q = (const float *)c->q_cur;
    float *gA = (float *)c->qgA, *gB = (float *)c->qgB;
    const bool second = c->cfg.order == 2;
    double best_q = 1e300, best_f = 1e300, def_q = 0.0, def_f = 0.0;
    int vq = 0, vf = 0;
    // q-derivative variants: one inner pass, reading the first-order gradient in gA
    lskum_status r = LSKUM_OK;
    if (LAUNCH_OK(c, launch_qgrad_mixed(g, q, nullptr, nullptr, gA, nullptr, 0.0, c->stream, 0), r)) {
        for (int v = 0; v < mixed_variants(1) && r == LSKUM_OK; ++v) {
            double ms = 0.0;
            r = time_variant(c, reps, e0, e1,
                             [&] { return launch_qgrad_mixed(g, q, gA, gA, gB, nullptr, 0.0, c->stream, v); }, &ms);
            if (v == 0) def_q = ms;
            if (r == LSKUM_OK && ms < best_q) { best_q = ms; vq = v; }
        }
    }
    // flux variants: residual mode into the scratch residual
    MixedFluxParams P{};
    P.g = g;
    P.nrm64 = c->nrm;
    P.q = q;
    P.qg = second ? gA : nullptr;
    P.Un = c->U;
    P.acc = c->acc;
    P.dt = c->dt;
    P.R = c->Rt;
    P.norm_part = c->norm_part;
    P.status = c->status;
    P.pcase = c->pcase;
    P.case_uinf = c->case_uinf;
    for (int k = 0; k < 4; ++k) P.Uinf[k] = c->gas.Uinf[k];
    P.gamma = (float)c->gas.gamma;
    P.inv_gm1 = (float)c->gas.inv_gm1;
    P.cfl = (float)c->cfg.cfl;
    P.g14 = c->gas.g14;
    P.order = c->cfg.order;
    P.mode = 0;
    for (int v = 0; v < mixed_variants(0) && r == LSKUM_OK; ++v) {
        double ms = 0.0;
        r = time_variant(c, reps, e0, e1, [&] { return launch_flux_mixed(P, c->stream, v); }, &ms);
        if (v == 0) def_f = ms;
        if (r == LSKUM_OK && ms < best_f) { best_f = ms; vf = v; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r != LSKUM_OK) return r;
    if ((st = check_nonphysical(c)) != LSKUM_OK) return st;
    c->var_flux = vf;
    c->var_qgrad = vq;
    drop_graphs(c);
    if (out) {
        out->flux_variant = vf;
        mixed_variant_shape(0, vf, &out->flux_threads, &out->flux_min_blocks);
        out->qgrad_variant = vq;
        mixed_variant_shape(1, vq, &out->qgrad_threads, &out->qgrad_min_blocks);
        out->flux_ms = best_f;
        out->qgrad_ms = best_q;
        out->flux_ms_default = def_f;
        out->qgrad_ms_default = def_q;
    }
    return LSKUM_OK;
}

extern "C" lskum_status lskum_case_forces(lskum_ctx *c, int k, double *cl, double *cd, double *cp)
{
    if (!c) return LSKUM_ERR_ARG;
    c->err.clear();
    if (!cl || !cd) return fail(c, LSKUM_ERR_ARG, "cl or cd is NULL");
    if (k < 0 || k >= c->ncases) return fail(c, LSKUM_ERR_ARG, "case %d out of range", k);
    const int64_t w0 = c->case_wall_h[k], nw = c->case_wall_h[k + 1] - w0;
    if (nw == 0) return fail(c, LSKUM_ERR_ARG, "no wall contour was given at create for case %d", k);
    const double a = c->case_aoa[k] * 3.14159265358979323846 / 180.0;
    const double qinf = 0.5 * c->case_mach[k] * c->case_mach[k];
    if (!(qinf > 0.0)) return fail(c, LSKUM_ERR_ARG, "forces need mach > 0");
    double *out = c->fbuf + c->n_wall + 2 * k;
    LAUNCH(c, launch_forces(nw, c->gas, qinf, c->wall + w0, c->wall_ds + w0, c->nrm, c->U, cos(a), sin(a),
                            c->fbuf + w0, out, c->stream));
    double clcd[2];
    CK(c, cudaMemcpyAsync(clcd, out, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (cp) CK(c, cudaMemcpyAsync(cp, c->fbuf + w0, nw * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    *cl = clcd[0];
    *cd = clcd[1];
    return LSKUM_OK;
}

extern "C" lskum_status lskum_forces(lskum_ctx *c, double *cl, double *cd, double *cp)
{
    if (!c) return LSKUM_ERR_ARG;
    if (c->ncases != 1) return fail(c, LSKUM_ERR_ARG, "a batch context reports forces per case (lskum_case_forces)");
    return lskum_case_forces(c, 0, cl, cd, cp);
}

extern "C" lskum_status lskum_get_state(lskum_ctx *c, double *U, int on_host)
{
    if (!c) return LSKUM_ERR_ARG;
    c->err.clear();
    if (!U) return fail(c, LSKUM_ERR_ARG, "U is NULL");
    double *dst = on_host ? c->Ucm : U;
    LAUNCH(c, launch_state_out(c->n, c->perm, c->U, dst, c->stream));
    if (on_host) {
        CK(c, cudaMemcpyAsync(U, c->Ucm, 4 * c->n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
    }
    return LSKUM_OK;
}

extern "C" lskum_status lskum_set_state(lskum_ctx *c, const double *U, int on_host)
{
    if (!c) return LSKUM_ERR_ARG;
    c->err.clear();
    if (!U) return fail(c, LSKUM_ERR_ARG, "U is NULL");
    const double *src = U;
    if (on_host) {
        CK(c, cudaMemcpyAsync(c->Ucm, U, 4 * c->n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        src = c->Ucm;
    }
    lskum_status st = reset_status(c);
    if (st != LSKUM_OK) return st;
    LAUNCH(c, launch_state_in(c->n, c->perm, src, c->U, c->stream));
    if ((st = refresh_q(c, c->U, c->q_cur)) != LSKUM_OK) return st;
    if (on_host) return check_nonphysical(c);
    return LSKUM_OK;
}

extern "C" lskum_status lskum_get_stencil_masks(lskum_ctx *c, uint8_t *mask)
{
    if (!c) return LSKUM_ERR_ARG;
    c->err.clear();
    if (!mask) return fail(c, LSKUM_ERR_ARG, "mask is NULL");
    uint8_t *tmp = nullptr;
    CK(c, cudaMallocAsync(&tmp, std::max<int64_t>(c->nnz, 1), c->stream));
    c->launches++;
    cudaError_t e = launch_mask_out(c->n, c->inv, c->off_in, c->off, c->mask, tmp, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(mask, tmp, c->nnz, cudaMemcpyDeviceToHost, c->stream);
    cudaFreeAsync(tmp, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    CK(c, e);
    return LSKUM_OK;
}

extern "C" lskum_status lskum_get_permutation(lskum_ctx *c, int32_t *perm)
{
    if (!c) return LSKUM_ERR_ARG;
    if (!perm) return fail(c, LSKUM_ERR_ARG, "perm is NULL");
    memcpy(perm, c->perm_h.data(), c->n * sizeof(int32_t));
    return LSKUM_OK;
}

extern "C" lskum_status lskum_profile(lskum_ctx *c, int enable)
{
    if (!c) return LSKUM_ERR_ARG;
    CK(c, c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize());
    c->profiling = enable != 0;
    c->ev_used = 0;
    for (auto &v : c->timed) v.clear();
    return LSKUM_OK;
}

extern "C" lskum_status lskum_kernel_time(lskum_ctx *c, int cls, double *total_ms, int64_t *launches)
{
    if (!c) return LSKUM_ERR_ARG;
    if (cls < 0 || cls >= LSKUM_KERNEL_CLASSES || !total_ms || !launches)
        return fail(c, LSKUM_ERR_ARG, "bad kernel class or output pointer");
    CK(c, c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize());
    double t = 0.0;
    for (auto &pr : c->timed[cls]) {
        float ms = 0.0f;
        CK(c, cudaEventElapsedTime(&ms, pr.first, pr.second));
        t += ms;
    }
    *total_ms = t;
    *launches = (int64_t)c->timed[cls].size();
    return LSKUM_OK;
}
