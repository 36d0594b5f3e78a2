// C ABI and host runtime of the B300 HPR-LP solver; declarations in include/hpr.h.
//
// Host responsibilities: validate the LP, assemble A = [A1; A2], build the explicit
// CSR of A^T (stable counting sort) and the sliced-ELL layouts of both matrices with
// their row / column renumbering (rows by decreasing length, stable), drive
// the preprocessing / power-method / iteration kernels, and take the scalar decisions
// of Algorithm 2 (termination, restart criteria of Section 3.1, Algorithm 3) once per
// check period from ~16 reduced FP64 scalars.  Every vector operation of the method
// runs in the kernels of hpr_device.cuh.
//
// Iteration schedule (same reading as the documentation of the method's oracle):
// iteration k (0-based) maps w^k to w^{k+1}; it is a check when (k+1) % check_every == 0
// or k+1 == max_iter, and evaluates R~_{r,0} when the inner counter t is 0.  Restarts
// happen only at checks, so every check period is one batch of iterations whose last
// iteration is a check and whose first is an R~_{r,0} evaluation right after a restart:
// the batch is captured once as a CUDA graph and replayed.
#include "hpr.h"
#include "hpr_device.cuh"
#include "hpr_mlp.cuh"
#include "hpr_small.cuh"

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <thread>
#include <type_traits>
#include <mutex>
#include <string>
#include <vector>

using namespace hprdev;

namespace {

struct GraphKey {
    int L;
    int first;
    int form;      // 0: FP64, 1: FP32 form
    bool operator<(const GraphKey &o) const
    {
        if (L != o.L) return L < o.L;
        if (first != o.first) return first < o.first;
        return form < o.form;
    }
};

}  // namespace


// one matrix in the sliced-ELL layout (device arrays; see k_sell)
struct SellDev {
    int rows = 0, nslices = 0;
    int64_t entries = 0;          // stored entries (nonzeros + padding)
    int steps_max = 0;            // layout parameters (build_sell)
    double unit_cost = 0.0;
    int nruns = 0;                // work units (one per warp)
    int grid = 0;                 // CTAs of a sliced-ELL launch: ceil(nruns / warps per CTA)
    int *srow = nullptr, *sptr = nullptr, *wstart = nullptr, *col = nullptr;
    unsigned char *slg = nullptr;
    std::vector<float> ucost;     // host: cost of each work unit (for batched work lists)
    double *val = nullptr;
    float *val32 = nullptr;       // FP32 copy of val (the FP32 form)
    int *src = nullptr;           // CSR position of each stored entry (-1: padding)
};

// state of a solve between its periods (Algorithm 2's counters and the last check)
struct SolveState {
    double tol = 1e-8, t0 = 0.0, lambda = 0.0, sigma = 1.0;
    int64_t k = 0, t = 0, r = 0;          // total, inner and outer counters
    int status = HPR_MAX_ITER;
    double R0 = 0.0, Rprev = 0.0;
    double last_pobj = 0, last_dobj = 0, last_ep = 0, last_ed = 0, last_gap = 0, last_kkt = 0;
    double time_1e4 = -1.0;
    int64_t iters_1e4 = -1, iters_fp32 = 0;
    bool tracing = false, done = false;
    bool ctl_off = false;                 // batched: the control block already says inactive
    int64_t policy_decisions = 0, policy_fallbacks = 0;
    bool policy_watch = false;            // a learned sigma is in use: watch the KKT residual
    bool policy_suspend = false;          // it rose: the next restart keeps Algorithm 3's sigma
    double policy_kkt = 0.0;              // KKT residual at the learned decision
    int L = 0;                            // the current period: iterations and whether it
    bool first_r0 = false;                // starts an inner loop (t = 0)
};

struct hpr_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t home_stream = nullptr;   // the context's own stream (a batch swaps `stream`)
    hpr_options opt{};
    int64_t m1 = 0, m2 = 0, m = 0, n = 0, nnz = 0;
    double norm_b = 0.0, norm_c = 0.0, beta_b = 1.0, beta_c = 1.0;

    // matrices (device): scaled A, its explicit transpose and the transpose map
    int *A_rp = nullptr, *A_ci = nullptr;
    double *A_val = nullptr;
    int *T_rp = nullptr, *T_ci = nullptr, *T_perm = nullptr;
    double *T_val = nullptr;
    SellDev SA, ST;               // A and A^T in the renumbered sliced-ELL layout
    int *perm_r = nullptr;        // renumbered row i of A is original row perm_r[i]
    int *perm_c = nullptr;        // renumbered column j is original column perm_c[j]
    unsigned char *ineq = nullptr;// renumbered row i belongs to A2 (m2 block)
    int num_sms = 0;

    // vectors (device)
    // preprocessing results in the original order
    double *Dr = nullptr, *Dc = nullptr, *wr = nullptr, *wc = nullptr;
    double *b_s = nullptr, *c_s = nullptr, *l_s = nullptr, *u_s = nullptr;
    double *l_o = nullptr, *u_o = nullptr;
    // the same in the renumbered order used by the iteration
    double *bp = nullptr, *cp = nullptr, *lp = nullptr, *up = nullptr, *wrp = nullptr, *wcp = nullptr;
    double *unperm = nullptr;     // n + m scratch for copying iterates out in the original order
    double *x = nullptr, *x0 = nullptr, *xhat = nullptr, *xbar = nullptr, *zbar = nullptr,
           *dx = nullptr;
    double *y = nullptr, *y0 = nullptr, *ybar = nullptr, *dy = nullptr;
    float *x32 = nullptr, *xhat32 = nullptr, *y32 = nullptr;   // FP32-form iterates
    int form = 0;                 // form of the iterates during a solve (0 FP64, 1 FP32)
    double *xo = nullptr, *yo = nullptr, *zo = nullptr;

    // reductions and control
    double *partials = nullptr;
    int pstride = 0;
    double *scal = nullptr;     // device, 2 slots of NQ
    double *scal_h = nullptr;   // pinned mirror
    DevCtl *ctl = nullptr;      // device control block
    DevCtl *ctl_h = nullptr;    // pinned staging
    size_t ctl_bytes = 0;
    int ctl_cap = 0;
    PowCtl *pctl = nullptr, *pctl_h = nullptr;
    double *trace = nullptr;
    int64_t trace_n = 0;
    int64_t trace_written = 0;

    std::map<GraphKey, cudaGraphExec_t> graphs;
    std::map<GraphKey, int64_t> graph_launches;   // kernel nodes per captured period
    cudaGraphExec_t pow_graph = nullptr;

    // host structure of the layouts that the small-phase rule gave short slices, kept so
    // that a batch whose fused phases move enough data can lay them out for throughput
    // (freed once it has)
    struct Relayout {
        bool a = false, t = false;               // A's / A^T's layout took the small-phase rule
        std::vector<int> rp, ci, pr, ipc;        // A: CSR, row order, column renaming
        std::vector<int> trp, tci, pc, ipr;      // A^T: the same
    };
    std::unique_ptr<Relayout> relayout;
    int64_t launches = 0;                           // kernels launched by the current solve

    // results
    bool solved = false;
    bool have_power = false;
    double lambda = 0.0;
    int64_t power_iters = 0;
    double power_time = 0.0;
    hpr_info info{};
    SolveState ss;
    __nv_bfloat16 *policy_wb = nullptr;   // sigma policy network (BF16), its input and output
    float *policy_w32 = nullptr, *policy_x = nullptr, *policy_q = nullptr;
    hpr_check_record *small_recs = nullptr;   // persistent path: its check records and results
    double *small_out = nullptr;
    int small_cap = 0;
    hprsmall::SmallArgs *small_args = nullptr; // persistent path: device copy of its arguments
    bool batched = false;         // owned by a batch: solved only through hpr_batch_solve
    std::vector<hpr_check_record> checks;
    std::string err;
};

namespace {

const char *g_static_err = "no context";

int fail_cuda(hpr_ctx *c, cudaError_t e, const char *what, int line)
{
    char buf[512];
    snprintf(buf, sizeof buf, "%s failed at line %d: %s (%s)", what, line, cudaGetErrorName(e),
             cudaGetErrorString(e));
    if (c) c->err = buf;
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? HPR_ERR_NOMEM : HPR_ERR_CUDA;
}

int fail_arg(hpr_ctx *c, int code, const std::string &msg)
{
    if (c) c->err = msg;
    return code;
}

#define CK(call)                                                                  \
    do {                                                                          \
        cudaError_t e_ = (call);                                                  \
        if (e_ != cudaSuccess) return fail_cuda(ctx, e_, #call, __LINE__);        \
    } while (0)

#define CKL()                                                                     \
    do {                                                                          \
        cudaError_t e_ = cudaGetLastError();                                      \
        if (e_ != cudaSuccess) return fail_cuda(ctx, e_, "kernel launch", __LINE__); \
    } while (0)

template <class T>
int dalloc(hpr_ctx *ctx, T **p, int64_t count)
{
    size_t bytes = sizeof(T) * (size_t)(count > 0 ? count : 1);
    cudaError_t e = cudaMalloc((void **)p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail_cuda(ctx, e, "cudaMalloc", __LINE__);
    }
    return HPR_OK;
}

#define DALLOC(p, cnt)                          \
    do {                                        \
        int s_ = dalloc(ctx, &(p), (cnt));      \
        if (s_ != HPR_OK) return s_;            \
    } while (0)

int grid_for(int64_t n, int threads = 256, int cap = 148 * 16)
{
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

// Renumbering by decreasing row length, stable (rows of equal length keep their order,
// so locality inside a length class survives): perm[new] = old.
std::vector<int> order_by_length(const std::vector<int> &rp, int rows)
{
    int maxlen = 0;
    for (int i = 0; i < rows; ++i) maxlen = std::max(maxlen, rp[(size_t)i + 1] - rp[(size_t)i]);
    std::vector<int> cnt((size_t)maxlen + 2, 0);
    for (int i = 0; i < rows; ++i) cnt[(size_t)(maxlen - (rp[(size_t)i + 1] - rp[(size_t)i]))]++;
    int acc = 0;
    for (auto &v : cnt) { const int c = v; v = acc; acc += c; }
    std::vector<int> perm((size_t)rows);
    for (int i = 0; i < rows; ++i) perm[(size_t)cnt[(size_t)(maxlen - (rp[(size_t)i + 1] - rp[(size_t)i]))]++] = i;
    return perm;
}

// Sliced-ELL layout of a CSR matrix (rows in the order perm, longest first; columns
// renamed by icol): host index arrays; the values are gathered on the GPU through `src`.
// Rows are taken in groups of 32; a group uses L lanes per row, L the smallest power of
// two that keeps its widest slice within `steps_max` steps (L <= 32), and is stored as L
// slices of 32 / L rows.  Work units (one per warp): a group whole, or each slice of a
// group whose cost exceeds `unit_cost`.  Defaults 40 and 64 (16 and 32 for phases below
// SMALL_PHASE_BYTES); the autotuner may pick others.
constexpr int SELL_STEPS = 40;
constexpr double UNIT_COST = 64.0;
constexpr double SMALL_PHASE_BYTES = 40e6;   // below: SMALL_SELL_STEPS and SMALL_UNIT_COST
constexpr int SMALL_SELL_STEPS = 16;
constexpr double SMALL_UNIT_COST = 32.0;

struct SellHost {
    int nslices = 0;
    std::vector<int> srow, sptr, col, src, wstart;
    std::vector<unsigned char> slg;
    std::vector<float> ucost;        // cost of each work unit (steps + epilogue share)
    int steps_max = SELL_STEPS;
    double unit_cost = UNIT_COST;
};

SellHost build_sell(const std::vector<int> &rp, const std::vector<int> &ci, int rows,
                    const std::vector<int> &perm, const std::vector<int> &icol,
                    int steps_max = SELL_STEPS, double unit_cost = UNIT_COST)
{
    SellHost h;
    h.steps_max = steps_max;
    h.unit_cost = unit_cost;
    auto len = [&](int i) { return rp[(size_t)perm[(size_t)i] + 1] - rp[(size_t)perm[(size_t)i]]; };
    std::vector<double> scost;       // cost of each slice (epilogue share included)
    std::vector<int> gfirst;         // first slice of each group
    h.srow.push_back(0);
    h.sptr.push_back(0);
    for (int g0 = 0; g0 < rows; g0 += 32) {
        const int g1 = std::min(rows, g0 + 32);
        const int lmax = len(g0);
        int lg = 0;
        while (lg < 5 && (lmax + (1 << lg) - 1) / (1 << lg) > steps_max) ++lg;
        const int L = 1 << lg, per = 32 / L;
        gfirst.push_back(h.nslices);
        for (int r = g0; r < g1; r += per) {
            const int r1 = std::min(g1, r + per);
            const int steps = (len(r) + L - 1) / L;
            const size_t base = h.col.size();
            h.col.resize(base + (size_t)32 * steps, 0);
            h.src.resize(base + (size_t)32 * steps, -1);
            for (int q = 0; q < r1 - r; ++q) {
                const int orow = perm[(size_t)(r + q)];
                for (int e = 0, p = rp[(size_t)orow]; p < rp[(size_t)orow + 1]; ++p, ++e) {
                    const size_t at = base + (size_t)(e / L) * 32 + (size_t)(q * L + e % L);
                    h.col[at] = icol[(size_t)ci[(size_t)p]];
                    h.src[at] = p;
                }
            }
            h.slg.push_back((unsigned char)lg);
            h.srow.push_back(r1);
            h.sptr.push_back((int)h.col.size());
            h.nslices++;
            scost.push_back((double)steps + 2.0 + lg + 8.0 * (r1 - r) / 32.0);
        }
    }
    gfirst.push_back(h.nslices);
    // work units: a light group whole, a heavy group by slice
    h.wstart.clear();
    for (size_t g = 0; g + 1 < gfirst.size(); ++g) {
        double gc = 0.0;
        for (int sl = gfirst[g]; sl < gfirst[g + 1]; ++sl) gc += scost[(size_t)sl];
        if (gc <= unit_cost) {
            h.wstart.push_back(gfirst[g]);
            h.ucost.push_back((float)gc);
        } else {
            for (int sl = gfirst[g]; sl < gfirst[g + 1]; ++sl) {
                h.wstart.push_back(sl);
                h.ucost.push_back((float)scost[(size_t)sl]);
            }
        }
    }
    h.wstart.push_back(h.nslices);
    return h;
}

int validate_block(hpr_ctx *ctx, const hpr_csr *B, const char *name, int64_t *rows, int64_t *cols)
{
    if (!B || B->rows == 0) {
        *rows = 0;
        *cols = B ? B->cols : -1;
        if (B && B->nnz != 0) return fail_arg(ctx, HPR_ERR_ARG, std::string(name) + ": rows = 0 but nnz != 0");
        return HPR_OK;
    }
    if (B->rows < 0 || B->cols < 0 || B->nnz < 0)
        return fail_arg(ctx, HPR_ERR_ARG, std::string(name) + ": negative size");
    if (B->rows >= (int64_t)INT32_MAX || B->cols >= (int64_t)INT32_MAX || B->nnz >= (int64_t)INT32_MAX)
        return fail_arg(ctx, HPR_ERR_ARG, std::string(name) + ": sizes beyond 2^31-1 are not supported");
    if (!B->row_ptr || (B->nnz > 0 && (!B->col_idx || !B->val)))
        return fail_arg(ctx, HPR_ERR_ARG, std::string(name) + ": NULL array");
    if (B->row_ptr[0] != 0 || B->row_ptr[B->rows] != B->nnz)
        return fail_arg(ctx, HPR_ERR_ARG, std::string(name) + ": row_ptr[0] != 0 or row_ptr[rows] != nnz");
    for (int64_t i = 0; i < B->rows; ++i) {
        const int64_t a = B->row_ptr[i], b = B->row_ptr[i + 1];
        if (b < a) return fail_arg(ctx, HPR_ERR_ARG, std::string(name) + ": row_ptr decreases");
        for (int64_t p = a; p < b; ++p) {
            const int32_t cidx = B->col_idx[p];
            if (cidx < 0 || cidx >= B->cols)
                return fail_arg(ctx, HPR_ERR_ARG, std::string(name) + ": column index out of range");
            if (p > a && cidx <= B->col_idx[p - 1])
                return fail_arg(ctx, HPR_ERR_ARG, std::string(name) + ": column indices not strictly increasing in a row");
            if (!std::isfinite(B->val[p]))
                return fail_arg(ctx, HPR_ERR_ARG, std::string(name) + ": non-finite value");
        }
    }
    *rows = B->rows;
    *cols = B->cols;
    return HPR_OK;
}

void free_all(hpr_ctx *c)
{
    if (!c) return;
    for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second);
    c->graphs.clear();
    if (c->pow_graph) cudaGraphExecDestroy(c->pow_graph);
    c->pow_graph = nullptr;
    void *dev[] = {c->A_rp, c->A_ci, c->A_val, c->T_rp, c->T_ci, c->T_perm, c->T_val,
                   c->SA.srow, c->SA.sptr, c->SA.wstart, c->SA.slg, c->SA.col, c->SA.val, c->SA.src,
                   c->ST.srow, c->ST.sptr, c->ST.wstart, c->ST.slg, c->ST.col, c->ST.val, c->ST.src,
                   c->SA.val32, c->ST.val32, c->x32, c->xhat32, c->y32,
                   c->perm_r, c->perm_c, c->ineq, c->bp, c->cp, c->lp, c->up, c->wrp, c->wcp,
                   c->unperm, c->Dr, c->Dc, c->wr, c->wc, c->b_s, c->c_s,
                   c->l_s, c->u_s, c->l_o, c->u_o, c->x, c->x0, c->xhat, c->xbar,
                   c->zbar, c->dx, c->y, c->y0, c->ybar, c->dy, c->xo, c->yo, c->zo,
                   c->partials, c->scal, c->ctl, c->pctl, c->trace, c->policy_wb, c->policy_w32,
                   c->policy_x, c->policy_q, c->small_recs, c->small_out, c->small_args};
    for (void *p : dev)
        if (p) cudaFree(p);
    if (c->scal_h) cudaFreeHost(c->scal_h);
    if (c->ctl_h) cudaFreeHost(c->ctl_h);
    if (c->pctl_h) cudaFreeHost(c->pctl_h);
    if (c->own_stream && c->home_stream) cudaStreamDestroy(c->home_stream);
}

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// ---------------------------------------------------------------- launches

int launch_reduce(hpr_ctx *ctx, const std::vector<std::pair<int, int>> &qc, double *out,
                  const int *skip = nullptr)
{
    RedSpec s{};
    s.nq = 0;
    for (auto &p : qc) {
        if (p.second <= 0) continue;
        s.q[s.nq] = p.first;
        s.cnt[s.nq] = p.second;
        s.nq++;
    }
    // quantities without any partial (empty side) are zero
    for (auto &p : qc)
        if (p.second <= 0) CK(cudaMemsetAsync(out + p.first, 0, sizeof(double), ctx->stream));
    if (s.nq == 0) return HPR_OK;
    k_reduce<<<s.nq, TB, 0, ctx->stream>>>(ctx->partials, ctx->pstride, s, out, skip);
    CKL();
    ctx->launches += 1;
    return HPR_OK;
}

SellArgs sell_of(const SellDev &d, bool fp32, const int *skip = nullptr)
{
    SellArgs a;
    a.rows = d.rows; a.nslices = d.nslices; a.srow = d.srow; a.sptr = d.sptr; a.slg = d.slg;
    a.wstart = d.wstart; a.nruns = d.nruns; a.col = d.col; a.skip = skip;
    a.val = fp32 ? (const void *)d.val32 : (const void *)d.val;
    a.trigger_from = INT32_MAX;
    return a;
}

// every k_sell instance must fit at least one CTA on an SM (its launch bounds)
template <class E>
int check_kernel(hpr_ctx *ctx)
{
    int per_sm = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sell<E>, SELL_TB, 0));
    if (per_sm < 1) return fail_arg(ctx, HPR_ERR_CUDA, "sliced-ELL kernel does not fit on an SM");
    return HPR_OK;
}

template <class E>
int launch_sell(hpr_ctx *ctx, const SellDev &M, const E &e, const int *skip = nullptr)
{
    if (M.rows == 0) return HPR_OK;
    k_sell<E><<<M.grid, SELL_TB, 0, ctx->stream>>>(sell_of(M, sizeof(typename E::Val) == 4, skip), e);
    CKL();
    ctx->launches += 1;
    return HPR_OK;
}

// a normal-iteration phase launched as a programmatic dependent of the kernel before it:
// the CTAs of its last wave (the ones resident at once) let the next phase launch early
template <class E>
int launch_sell_pdl(hpr_ctx *ctx, const SellDev &M, const E &e)
{
    if (M.rows == 0) return HPR_OK;
    if (!ctx->opt.pdl) return launch_sell(ctx, M, e);
    SellArgs a = sell_of(M, sizeof(typename E::Val) == 4);
    a.trigger_from = std::max(0, M.grid - SELL_CTAS_PER_SM * ctx->num_sms);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)M.grid);
    cfg.blockDim = dim3(SELL_TB);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CK(cudaLaunchKernelEx(&cfg, k_sell<E>, a, e));
    ctx->launches += 1;
    return HPR_OK;
}

template <bool CHECK>
EpiX<CHECK> epi_x(hpr_ctx *c, int it)
{
    EpiX<CHECK> e{};
    e.xa = c->y; e.xb = c->y;
    e.q[0] = Q_DX2; e.q[1] = Q_XX0; e.q[2] = Q_CX; e.q[3] = Q_BND;
    e.partials = c->partials; e.pstride = c->pstride;
    e.c = c->cp; e.l = c->lp; e.u = c->up; e.x0 = c->x0;
    e.x = c->x; e.xhat = c->xhat; e.xbar = c->xbar; e.zbar = c->zbar; e.dx = c->dx;
    e.ctl = c->ctl; e.it = it; e.reflect = (int)c->opt.reflect;
    return e;
}

template <bool CHECK>
EpiY<CHECK> epi_y(hpr_ctx *c, int it)
{
    EpiY<CHECK> e{};
    e.xa = c->xhat; e.xb = c->xhat;
    e.q[0] = Q_DY2; e.q[1] = Q_YY0; e.q[2] = Q_BY;
    e.partials = c->partials; e.pstride = c->pstride;
    e.b = c->bp; e.y0 = c->y0; e.y = c->y; e.ybar = c->ybar; e.dy = c->dy;
    e.ctl = c->ctl; e.it = it; e.ineq = c->ineq; e.reflect = (int)c->opt.reflect;
    return e;
}

template <bool CHECK>
EpiX32<CHECK> epi_x32(hpr_ctx *c, int it)
{
    EpiX32<CHECK> e{};
    e.xa = c->y32; e.xb = c->y32;
    e.q[0] = Q_DX2; e.q[1] = Q_XX0; e.q[2] = Q_CX; e.q[3] = Q_BND;
    e.partials = c->partials; e.pstride = c->pstride;
    e.c = c->cp; e.l = c->lp; e.u = c->up; e.x0 = c->x0;
    e.x = c->x32; e.xhat = c->xhat32; e.xbar = c->xbar; e.zbar = c->zbar; e.dx = c->dx;
    e.ctl = c->ctl; e.it = it; e.reflect = (int)c->opt.reflect;
    return e;
}

template <bool CHECK>
EpiY32<CHECK> epi_y32(hpr_ctx *c, int it)
{
    EpiY32<CHECK> e{};
    e.xa = c->xhat32; e.xb = c->xhat32;
    e.q[0] = Q_DY2; e.q[1] = Q_YY0; e.q[2] = Q_BY;
    e.partials = c->partials; e.pstride = c->pstride;
    e.b = c->bp; e.y0 = c->y0; e.y = c->y32; e.ybar = c->ybar; e.dy = c->dy;
    e.ctl = c->ctl; e.it = it; e.ineq = c->ineq; e.reflect = (int)c->opt.reflect;
    return e;
}

EpiNorm epi_norm(hpr_ctx *c, const double *xin, double *out, int q)
{
    EpiNorm e{};
    e.xa = xin; e.xb = xin; e.q[0] = q; e.partials = c->partials; e.pstride = c->pstride; e.out = out;
    return e;
}

// residual passes of a check: dual (A^T y_bar) and primal with the M-norm cross term (A x_bar, A dx)
EpiDual epi_dual(hpr_ctx *ctx)
{
    EpiDual d{};
    d.xa = ctx->ybar; d.xb = ctx->ybar; d.q[0] = Q_RD;
    d.partials = ctx->partials; d.pstride = ctx->pstride;
    d.c = ctx->cp; d.zbar = ctx->zbar; d.wc = ctx->wcp;
    d.ctl = ctx->ctl; d.it = 0;
    return d;
}

EpiPrimal epi_primal(hpr_ctx *ctx)
{
    EpiPrimal p{};
    p.xa = ctx->xbar; p.xb = ctx->dx; p.q[0] = Q_RP; p.q[1] = Q_CROSS;
    p.partials = ctx->partials; p.pstride = ctx->pstride;
    p.b = ctx->bp; p.wr = ctx->wrp; p.dy = ctx->dy; p.ineq = ctx->ineq;
    p.ctl = ctx->ctl; p.it = 0;
    return p;
}

// one HPR iteration (phase X then phase Y).  store: the phases also store x_bar, z_bar,
// y_bar, x - x_bar, y - y_bar; check: the two residual passes run and every check
// quantity is reduced into scal slot `slot`.
int enqueue_iteration(hpr_ctx *ctx, int it, bool store, bool check, int slot)
{
    int st;
    if (ctx->form == 1) {
        if (store || check) {
            if ((st = launch_sell(ctx, ctx->ST, epi_x32<true>(ctx, it)))) return st;
            if ((st = launch_sell(ctx, ctx->SA, epi_y32<true>(ctx, it)))) return st;
        } else {
            if ((st = launch_sell_pdl(ctx, ctx->ST, epi_x32<false>(ctx, it)))) return st;
            if ((st = launch_sell_pdl(ctx, ctx->SA, epi_y32<false>(ctx, it)))) return st;
        }
    } else if (store || check) {
        if ((st = launch_sell(ctx, ctx->ST, epi_x<true>(ctx, it)))) return st;
        if ((st = launch_sell(ctx, ctx->SA, epi_y<true>(ctx, it)))) return st;
    } else {
        if ((st = launch_sell_pdl(ctx, ctx->ST, epi_x<false>(ctx, it)))) return st;
        if ((st = launch_sell_pdl(ctx, ctx->SA, epi_y<false>(ctx, it)))) return st;
    }
    if (!check) return HPR_OK;
    if ((st = launch_sell(ctx, ctx->ST, epi_dual(ctx)))) return st;
    if ((st = launch_sell(ctx, ctx->SA, epi_primal(ctx)))) return st;
    const int nX = ctx->ST.rows ? ctx->ST.grid : 0, nY = ctx->SA.rows ? ctx->SA.grid : 0;
    const int nD = nX, nP = nY;
    return launch_reduce(ctx, {{Q_DX2, nX}, {Q_XX0, nX}, {Q_CX, nX}, {Q_BND, nX},
                               {Q_DY2, nY}, {Q_YY0, nY}, {Q_BY, nY}, {Q_RD, nD},
                               {Q_RP, nP}, {Q_CROSS, nP}},
                         ctx->scal + slot * NQ);
}

int enqueue_period(hpr_ctx *ctx, int L, bool first_r0)
{
    for (int i = 0; i < L; ++i) {
        const bool last = (i == L - 1);
        const bool r0 = (i == 0 && first_r0);
        int s = enqueue_iteration(ctx, i, last || r0, last || r0, last ? 1 : 0);
        if (s != HPR_OK) return s;
    }
    return HPR_OK;
}

int trace_copy(hpr_ctx *ctx, int64_t k)
{
    if (k >= ctx->trace_n) return HPR_OK;
    const int64_t n = ctx->n, m = ctx->m;
    double *rec = ctx->trace + (size_t)k * (size_t)(3 * n + 2 * m);
    CK(cudaMemcpyAsync(rec, ctx->xbar, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(rec + 3 * n, ctx->ybar, sizeof(double) * m, cudaMemcpyDeviceToDevice, ctx->stream));
    if (ctx->form == 1) {
        // FP32-form iterates, widened into the record
        k_widen<<<grid_for(2 * n), 256, 0, ctx->stream>>>((int)n, (int)n, ctx->xhat32, ctx->x32, rec + n, rec + 2 * n);
        CKL();
        k_widen<<<grid_for(m), 256, 0, ctx->stream>>>(0, (int)m, ctx->x32, ctx->y32, nullptr, rec + 3 * n + m);
        CKL();
    } else {
        CK(cudaMemcpyAsync(rec + n, ctx->xhat, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
        CK(cudaMemcpyAsync(rec + 2 * n, ctx->x, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
        CK(cudaMemcpyAsync(rec + 3 * n + m, ctx->y, sizeof(double) * m, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    ctx->trace_written = std::max(ctx->trace_written, k + 1);
    return HPR_OK;
}

int ensure_ctl(hpr_ctx *ctx, int cap)
{
    if (cap <= ctx->ctl_cap) return HPR_OK;
    if (ctx->ctl) cudaFree(ctx->ctl);
    if (ctx->ctl_h) cudaFreeHost(ctx->ctl_h);
    ctx->ctl = nullptr;
    ctx->ctl_h = nullptr;
    for (auto &kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
    ctx->graphs.clear();
    ctx->ctl_bytes = sizeof(DevCtl) + sizeof(double) * 2 * (size_t)cap;
    CK(cudaMalloc((void **)&ctx->ctl, ctx->ctl_bytes));
    CK(cudaMallocHost((void **)&ctx->ctl_h, ctx->ctl_bytes));
    memset(ctx->ctl_h, 0, ctx->ctl_bytes);
    ctx->ctl_cap = cap;
    return HPR_OK;
}

// ---------------------------------------------------------------- power method

int run_power(hpr_ctx *ctx)
{
    const int64_t m = ctx->m;
    const int gm = (int)((m + TB - 1) / TB);
    // u (m) in dy, s = A^T u (n) in dx, w = A s (m) in ybar
    double *u = ctx->dy, *s = ctx->dx, *w = ctx->ybar;
    k_pow_start<<<gm, TB, 0, ctx->stream>>>((int)m, ctx->opt.seed, ctx->perm_r, u, ctx->partials,
                                             ctx->pstride);
    CKL();
    int st = launch_reduce(ctx, {{Q_V2, gm}}, ctx->scal);
    if (st) return st;
    double *invp = ctx->scal + Q_V2B;
    k_inv_sqrt_scalar<<<1, 1, 0, ctx->stream>>>(ctx->scal, Q_V2, invp);
    CKL();
    k_scale_vec<<<grid_for(m), 256, 0, ctx->stream>>>((int)m, u, u, nullptr, invp);
    CKL();

    PowCtl pc{};
    pc.tol = ctx->opt.power_tol;
    pc.max_iter = (int)std::max<int64_t>(1, ctx->opt.power_max_iter);
    *ctx->pctl_h = pc;
    CK(cudaMemcpyAsync(ctx->pctl, ctx->pctl_h, sizeof(PowCtl), cudaMemcpyHostToDevice, ctx->stream));

    auto enqueue_steps = [&](int steps) -> int {
        for (int k = 0; k < steps; ++k) {
            int r = launch_sell(ctx, ctx->ST, epi_norm(ctx, u, s, Q_S2), &ctx->pctl->done);
            if (r) return r;
            r = launch_reduce(ctx, {{Q_S2, ctx->ST.rows ? ctx->ST.grid : 0}}, ctx->scal, &ctx->pctl->done);
            if (r) return r;
            k_pow_after_s<<<1, 1, 0, ctx->stream>>>(ctx->pctl, ctx->scal);
            CKL();
            r = launch_sell(ctx, ctx->SA, epi_norm(ctx, s, w, Q_W2), &ctx->pctl->done);
            if (r) return r;
            r = launch_reduce(ctx, {{Q_W2, ctx->SA.rows ? ctx->SA.grid : 0}}, ctx->scal, &ctx->pctl->done);
            if (r) return r;
            k_pow_after_w<<<1, 1, 0, ctx->stream>>>(ctx->pctl, ctx->scal);
            CKL();
            k_scale_vec<<<grid_for(m), 256, 0, ctx->stream>>>((int)m, w, u, ctx->pctl, nullptr);
            CKL();
            k_pow_finish<<<1, 1, 0, ctx->stream>>>(ctx->pctl);
            CKL();
        }
        return HPR_OK;
    };

    const int BATCH = 16;
    if (ctx->opt.use_graph && !ctx->pow_graph) {
        cudaGraph_t g;
        CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        const int64_t before = ctx->launches;
        int r = enqueue_steps(BATCH);
        ctx->launches = before;
        cudaGraph_t gg = nullptr;
        cudaError_t e = cudaStreamEndCapture(ctx->stream, &gg);
        if (r) { if (gg) cudaGraphDestroy(gg); return r; }
        if (e != cudaSuccess) return fail_cuda(ctx, e, "cudaStreamEndCapture", __LINE__);
        g = gg;
        e = cudaGraphInstantiate(&ctx->pow_graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail_cuda(ctx, e, "cudaGraphInstantiate", __LINE__);
    }
    ctx->launches += 3;   // start vector, 1/norm, normalisation (+1 for the reduction above)
    for (int64_t done_steps = 0; done_steps <= ctx->opt.power_max_iter; done_steps += BATCH) {
        if (ctx->opt.use_graph) {
            ctx->launches += (int64_t)BATCH * 8;
            CK(cudaGraphLaunch(ctx->pow_graph, ctx->stream));
        } else {
            ctx->launches += (int64_t)BATCH * 4;   // the 2 SpMVs and 2 reductions count themselves
            int r = enqueue_steps(BATCH);
            if (r) return r;
        }
        CK(cudaMemcpyAsync(ctx->pctl_h, ctx->pctl, sizeof(PowCtl), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        if (ctx->pctl_h->done) break;
    }
    ctx->lambda = ctx->pctl_h->lam;
    ctx->power_iters = ctx->pctl_h->k;
    if (!std::isfinite(ctx->lambda) || !(ctx->lambda > 0.0))
        return fail_arg(ctx, HPR_ERR_NUMERIC, "power method returned a non-positive lambda");
    return HPR_OK;
}

// ---------------------------------------------------------------- create helpers

void free_layout(SellDev &D)
{
    void *p[] = {D.srow, D.sptr, D.wstart, D.slg, D.col, D.val, D.val32, D.src};
    for (void *q : p)
        if (q) cudaFree(q);
    D.srow = D.sptr = D.wstart = D.col = D.src = nullptr;
    D.slg = nullptr;
    D.val = nullptr;
    D.val32 = nullptr;
}

// device copy of a host layout, with values gathered from the scaled CSR values
int install_layout(hpr_ctx *ctx, SellDev &D, const SellHost &H, int rows, const double *csr_val)
{
    cudaStream_t s = ctx->stream;
    free_layout(D);
    D.rows = rows; D.nslices = H.nslices;
    D.steps_max = H.steps_max; D.unit_cost = H.unit_cost;
    D.nruns = (int)H.wstart.size() - 1;
    D.ucost = H.ucost;
    D.grid = std::max(1, (D.nruns + SELL_WARPS - 1) / SELL_WARPS);
    D.entries = (int64_t)H.col.size();
    DALLOC(D.val32, D.entries);
    DALLOC(D.srow, (int64_t)H.srow.size()); DALLOC(D.sptr, (int64_t)H.sptr.size());
    DALLOC(D.wstart, (int64_t)H.wstart.size()); DALLOC(D.slg, (int64_t)H.slg.size());
    DALLOC(D.col, D.entries); DALLOC(D.val, D.entries); DALLOC(D.src, D.entries);
    CK(cudaMemcpyAsync(D.srow, H.srow.data(), sizeof(int) * H.srow.size(), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(D.sptr, H.sptr.data(), sizeof(int) * H.sptr.size(), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(D.wstart, H.wstart.data(), sizeof(int) * H.wstart.size(), cudaMemcpyHostToDevice, s));
    if (!H.slg.empty()) CK(cudaMemcpyAsync(D.slg, H.slg.data(), H.slg.size(), cudaMemcpyHostToDevice, s));
    if (D.entries) {
        CK(cudaMemcpyAsync(D.col, H.col.data(), sizeof(int) * H.col.size(), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(D.src, H.src.data(), sizeof(int) * H.src.size(), cudaMemcpyHostToDevice, s));
        k_gather_src<<<grid_for(D.entries), 256, 0, s>>>(D.entries, csr_val, D.src, D.val); CKL();
        k_narrow<<<grid_for(D.entries), 256, 0, s>>>(D.entries, D.val, D.val32); CKL();
    }
    CK(cudaStreamSynchronize(s));
    return HPR_OK;
}

// average duration (ms) of a plain phase launch with the current layout: 2 launches to
// warm up, then 5 back to back between CUDA events (the values do not change the timing)
int time_phase(hpr_ctx *ctx, bool transpose, double *ms)
{
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    int st = HPR_OK;
    for (int r = 0; r < 7 && st == HPR_OK; ++r) {
        if (r == 2) cudaEventRecord(e0, ctx->stream);
        st = transpose ? launch_sell(ctx, ctx->ST, epi_x<false>(ctx, 0)) : launch_sell(ctx, ctx->SA, epi_y<false>(ctx, 0));
    }
    cudaEventRecord(e1, ctx->stream);
    cudaError_t e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (st == HPR_OK && e == cudaSuccess) cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    if (e != cudaSuccess) return fail_cuda(ctx, e, "time_phase", __LINE__);
    *ms = t / 5.0;
    return HPR_OK;
}

// The autotuner: for one matrix (A: the y phase, A^T: the x phase) time the phase kernel
// with the layout built for each lanes-per-row bound (steps_max 16 ... 128), then each unit
// size (unit_cost 32 ... 256) at the best bound, and keep the fastest layout (a candidate
// replaces the incumbent only when at least 2% faster).  Runs at creation, before any
// solve; the iterate vectors are zeroed first.
int autotune_layout(hpr_ctx *ctx, bool transpose, const std::vector<int> &rp, const std::vector<int> &ci,
                    const std::vector<int> &perm, const std::vector<int> &icol)
{
    SellDev &D = transpose ? ctx->ST : ctx->SA;
    if (D.rows == 0) return HPR_OK;
    const int rows = D.rows;
    const double *csr_val = transpose ? ctx->T_val : ctx->A_val;
    cudaStream_t s = ctx->stream;
    CK(cudaMemsetAsync(ctx->x, 0, sizeof(double) * ctx->n, s));
    CK(cudaMemsetAsync(ctx->x0, 0, sizeof(double) * ctx->n, s));
    CK(cudaMemsetAsync(ctx->xhat, 0, sizeof(double) * ctx->n, s));
    CK(cudaMemsetAsync(ctx->y, 0, sizeof(double) * ctx->m, s));
    CK(cudaMemsetAsync(ctx->y0, 0, sizeof(double) * ctx->m, s));
    CK(cudaMemcpyAsync(ctx->ctl, ctx->ctl_h, ctx->ctl_bytes, cudaMemcpyHostToDevice, s));
    int best_steps = D.steps_max;
    double best_cost = D.unit_cost, best_ms = 0.0;
    int st = time_phase(ctx, transpose, &best_ms);
    if (st) return st;
    auto trial = [&](int steps, double cost) -> int {
        if (steps == best_steps && cost == best_cost) return HPR_OK;
        SellHost H = build_sell(rp, ci, rows, perm, icol, steps, cost);
        int r = install_layout(ctx, D, H, rows, csr_val);
        if (r) return r;
        double ms = 0.0;
        if ((r = time_phase(ctx, transpose, &ms))) return r;
        if (ms < 0.98 * best_ms) {
            best_ms = ms;
            best_steps = steps;
            best_cost = cost;
        }
        return HPR_OK;
    };
    for (int steps : {16, 24, 40, 64, 128})
        if ((st = trial(steps, best_cost))) return st;
    for (double cost : {32.0, 64.0, 128.0, 256.0})
        if ((st = trial(best_steps, cost))) return st;
    if (D.steps_max != best_steps || D.unit_cost != best_cost) {
        SellHost H = build_sell(rp, ci, rows, perm, icol, best_steps, best_cost);
        if ((st = install_layout(ctx, D, H, rows, csr_val))) return st;
    }
    // the partial sums of the check kernels need one slot per CTA of the larger grid
    const int need = std::max(ctx->SA.grid, ctx->ST.grid);
    if (need > ctx->pstride) {
        cudaFree(ctx->partials);
        ctx->partials = nullptr;
        ctx->pstride = need;
        DALLOC(ctx->partials, (int64_t)NQ * ctx->pstride);
    }
    return HPR_OK;
}

// algorithmic bytes of the x phase (A^T) and the y phase (A) of one iteration
double phase_bytes_x(const hpr_ctx *c)
{
    return 12.0 * (double)c->nnz + 60.0 * (double)c->n + 8.0 * (double)c->m;
}

double phase_bytes_y(const hpr_ctx *c)
{
    return 12.0 * (double)c->nnz + 8.0 * (double)c->n + 36.0 * (double)c->m;
}

int upload_and_prepare(hpr_ctx *ctx, const hpr_csr *A1, const hpr_csr *A2, const double *b1,
                       const double *b2, const double *c, const double *l, const double *u)
{
    const int64_t m1 = ctx->m1, m2 = ctx->m2, m = ctx->m, n = ctx->n, nnz = ctx->nnz;

    // assemble A = [A1; A2] with 32-bit offsets
    std::vector<int> rp((size_t)m + 1);
    std::vector<int> ci((size_t)std::max<int64_t>(nnz, 1));
    std::vector<double> val((size_t)std::max<int64_t>(nnz, 1));
    int64_t off = 0;
    rp[0] = 0;
    const hpr_csr *blk[2] = {A1, A2};
    const int64_t brows[2] = {m1, m2};
    int64_t row = 0;
    for (int bI = 0; bI < 2; ++bI) {
        const hpr_csr *B = blk[bI];
        for (int64_t i = 0; i < brows[bI]; ++i, ++row) {
            for (int64_t p = B->row_ptr[i]; p < B->row_ptr[i + 1]; ++p, ++off) {
                ci[(size_t)off] = B->col_idx[p];
                val[(size_t)off] = B->val[p];
            }
            rp[(size_t)row + 1] = (int)off;
        }
    }
    // explicit CSR of A^T by a stable counting sort (rows of A^T list the rows of A in
    // increasing order) and the map from A^T positions to A positions
    std::vector<int> trp((size_t)n + 1, 0), tci((size_t)std::max<int64_t>(nnz, 1)),
        tperm((size_t)std::max<int64_t>(nnz, 1));
    for (int64_t p = 0; p < nnz; ++p) trp[(size_t)ci[(size_t)p] + 1]++;
    for (int64_t j = 0; j < n; ++j) trp[(size_t)j + 1] += trp[(size_t)j];
    {
        std::vector<int> next(trp.begin(), trp.end() - 1);
        for (int64_t i = 0; i < m; ++i)
            for (int p = rp[(size_t)i]; p < rp[(size_t)i + 1]; ++p) {
                const int q = next[(size_t)ci[(size_t)p]]++;
                tci[(size_t)q] = (int)i;
                tperm[(size_t)q] = p;
            }
    }
    // renumbering and sliced-ELL layouts of A (rows by length) and A^T (columns by length)
    std::vector<int> pr = order_by_length(rp, (int)m), pc = order_by_length(trp, (int)n);
    std::vector<int> ipr((size_t)m), ipc((size_t)n);
    for (int64_t i = 0; i < m; ++i) ipr[(size_t)pr[(size_t)i]] = (int)i;
    for (int64_t j = 0; j < n; ++j) ipc[(size_t)pc[(size_t)j]] = (int)j;
    const hpr_options &op = ctx->opt;
    // A phase that moves little data is bound by its longest work unit's chain of dependent
    // loads, not by bandwidth: below SMALL_PHASE_BYTES of algorithmic traffic the default
    // layout takes shorter slices and smaller units (measured on the QAP LP at N = 20: the
    // x phase 19.5 -> 10.3 us; the medium LP, at 95 / 74 MB a phase, gains nothing).
    const bool smallA = phase_bytes_y(ctx) < SMALL_PHASE_BYTES, smallT = phase_bytes_x(ctx) < SMALL_PHASE_BYTES;
    const int stepsA = op.sell_steps_a > 0 ? (int)op.sell_steps_a : (smallA ? SMALL_SELL_STEPS : SELL_STEPS);
    const int stepsT = op.sell_steps_t > 0 ? (int)op.sell_steps_t : (smallT ? SMALL_SELL_STEPS : SELL_STEPS);
    const double costA = op.unit_cost_a > 0.0 ? op.unit_cost_a : (smallA ? SMALL_UNIT_COST : UNIT_COST);
    const double costT = op.unit_cost_t > 0.0 ? op.unit_cost_t : (smallT ? SMALL_UNIT_COST : UNIT_COST);
    SellHost hA = build_sell(rp, ci, (int)m, pr, ipc, stepsA, costA);
    SellHost hT = build_sell(trp, tci, (int)n, pc, ipr, stepsT, costT);
    std::vector<unsigned char> ineq((size_t)m);
    for (int64_t i = 0; i < m; ++i) ineq[(size_t)i] = pr[(size_t)i] >= m1 ? 1 : 0;
    {
        int r;
        if ((r = check_kernel<EpiX<false>>(ctx))) return r;
        if ((r = check_kernel<EpiX<true>>(ctx))) return r;
        if ((r = check_kernel<EpiY<false>>(ctx))) return r;
        if ((r = check_kernel<EpiY<true>>(ctx))) return r;
        if ((r = check_kernel<EpiDual>(ctx))) return r;
        if ((r = check_kernel<EpiPrimal>(ctx))) return r;
        if ((r = check_kernel<EpiNorm>(ctx))) return r;
        if ((r = check_kernel<EpiX32<false>>(ctx))) return r;
        if ((r = check_kernel<EpiX32<true>>(ctx))) return r;
        if ((r = check_kernel<EpiY32<false>>(ctx))) return r;
        if ((r = check_kernel<EpiY32<true>>(ctx))) return r;
    }
    const int unitsA = (int)hA.wstart.size() - 1, unitsT = (int)hT.wstart.size() - 1;
    const int gA = std::max(1, (unitsA + SELL_WARPS - 1) / SELL_WARPS);
    const int gT = std::max(1, (unitsT + SELL_WARPS - 1) / SELL_WARPS);
    ctx->pstride = std::max({gA, gT, (int)((std::max(m, n) + TB - 1) / TB), 1});
    auto upload_sell = [&](SellDev &D, const SellHost &H, int rows) -> int {
        D.rows = rows; D.nslices = H.nslices;
        D.steps_max = H.steps_max; D.unit_cost = H.unit_cost;
        D.nruns = (int)H.wstart.size() - 1;
        D.ucost = H.ucost;
        D.grid = std::max(1, (D.nruns + SELL_WARPS - 1) / SELL_WARPS);
        D.entries = (int64_t)H.col.size();
        DALLOC(D.val32, D.entries);
        DALLOC(D.srow, (int64_t)H.srow.size()); DALLOC(D.sptr, (int64_t)H.sptr.size());
        DALLOC(D.wstart, (int64_t)H.wstart.size()); DALLOC(D.slg, (int64_t)H.slg.size());
        DALLOC(D.col, D.entries); DALLOC(D.val, D.entries); DALLOC(D.src, D.entries);
        CK(cudaMemcpyAsync(D.srow, H.srow.data(), sizeof(int) * H.srow.size(), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(D.sptr, H.sptr.data(), sizeof(int) * H.sptr.size(), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(D.wstart, H.wstart.data(), sizeof(int) * H.wstart.size(), cudaMemcpyHostToDevice, ctx->stream));
        if (!H.slg.empty())
            CK(cudaMemcpyAsync(D.slg, H.slg.data(), H.slg.size(), cudaMemcpyHostToDevice, ctx->stream));
        if (D.entries) {
            CK(cudaMemcpyAsync(D.col, H.col.data(), sizeof(int) * H.col.size(), cudaMemcpyHostToDevice, ctx->stream));
            CK(cudaMemcpyAsync(D.src, H.src.data(), sizeof(int) * H.src.size(), cudaMemcpyHostToDevice, ctx->stream));
        }
        return HPR_OK;
    };

    int st0;
    DALLOC(ctx->A_rp, m + 1); DALLOC(ctx->A_ci, nnz); DALLOC(ctx->A_val, nnz);
    DALLOC(ctx->T_rp, n + 1); DALLOC(ctx->T_ci, nnz); DALLOC(ctx->T_perm, nnz); DALLOC(ctx->T_val, nnz);
    if ((st0 = upload_sell(ctx->SA, hA, (int)m))) return st0;
    if ((st0 = upload_sell(ctx->ST, hT, (int)n))) return st0;
    DALLOC(ctx->perm_r, m); DALLOC(ctx->perm_c, n); DALLOC(ctx->ineq, m);

    DALLOC(ctx->bp, m); DALLOC(ctx->wrp, m); DALLOC(ctx->cp, n); DALLOC(ctx->lp, n); DALLOC(ctx->up, n);
    DALLOC(ctx->wcp, n); DALLOC(ctx->unperm, n + m);
    DALLOC(ctx->x32, n); DALLOC(ctx->xhat32, n); DALLOC(ctx->y32, m);
    DALLOC(ctx->Dr, m); DALLOC(ctx->Dc, n); DALLOC(ctx->wr, m); DALLOC(ctx->wc, n);
    DALLOC(ctx->b_s, m); DALLOC(ctx->c_s, n); DALLOC(ctx->l_s, n); DALLOC(ctx->u_s, n);
    DALLOC(ctx->l_o, n); DALLOC(ctx->u_o, n);
    DALLOC(ctx->x, n); DALLOC(ctx->x0, n); DALLOC(ctx->xhat, n); DALLOC(ctx->xbar, n);
    DALLOC(ctx->zbar, n); DALLOC(ctx->dx, n);
    DALLOC(ctx->y, m); DALLOC(ctx->y0, m); DALLOC(ctx->ybar, m); DALLOC(ctx->dy, m);
    DALLOC(ctx->xo, n); DALLOC(ctx->yo, m); DALLOC(ctx->zo, n);
    DALLOC(ctx->partials, (int64_t)NQ * ctx->pstride);
    DALLOC(ctx->scal, 2 * NQ);
    DALLOC(ctx->pctl, 1);
    CK(cudaMallocHost((void **)&ctx->scal_h, sizeof(double) * 2 * NQ));
    CK(cudaMallocHost((void **)&ctx->pctl_h, sizeof(PowCtl)));
    int st = ensure_ctl(ctx, (int)std::min<int64_t>(ctx->opt.check_every, ctx->opt.max_iter));
    if (st) return st;

    cudaStream_t s = ctx->stream;
    CK(cudaMemcpyAsync(ctx->A_rp, rp.data(), sizeof(int) * (m + 1), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->A_ci, ci.data(), sizeof(int) * nnz, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->A_val, val.data(), sizeof(double) * nnz, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->T_rp, trp.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->T_ci, tci.data(), sizeof(int) * nnz, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->T_perm, tperm.data(), sizeof(int) * nnz, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->perm_r, pr.data(), sizeof(int) * m, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->perm_c, pc.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->ineq, ineq.data(), m, cudaMemcpyHostToDevice, s));
    if (m1) CK(cudaMemcpyAsync(ctx->b_s, b1, sizeof(double) * m1, cudaMemcpyHostToDevice, s));
    if (m2) CK(cudaMemcpyAsync(ctx->b_s + m1, b2, sizeof(double) * m2, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->c_s, c, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->l_s, l, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->u_s, u, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->l_o, l, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->u_o, u, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));   // host staging vectors go out of scope below

    // ---- preprocessing of Section 4.1 (all on the GPU)
    const int gm = grid_for(m), gn = grid_for(n), gz = grid_for(nnz);
    k_fill<<<gm, 256, 0, s>>>(m, 1.0, ctx->Dr); CKL();
    k_fill<<<gn, 256, 0, s>>>(n, 1.0, ctx->Dc); CKL();
    double *dr = ctx->dy, *dc = ctx->dx;   // scratch
    for (int64_t it = 0; it < ctx->opt.ruiz_iters; ++it) {
        k_gather<<<gz, 256, 0, s>>>(nnz, ctx->A_val, ctx->T_perm, ctx->T_val); CKL();
        k_row_absmax<<<gm, 256, 0, s>>>((int)m, ctx->A_rp, ctx->A_val, dr); CKL();
        k_row_absmax<<<gn, 256, 0, s>>>((int)n, ctx->T_rp, ctx->T_val, dc); CKL();
        k_factor<<<gm, 256, 0, s>>>((int)m, dr, ctx->Dr); CKL();
        k_factor<<<gn, 256, 0, s>>>((int)n, dc, ctx->Dc); CKL();
        k_scale_rows_cols<<<gm, 256, 0, s>>>((int)m, ctx->A_rp, ctx->A_ci, ctx->A_val, dr, dc); CKL();
    }
    if (ctx->opt.pc_alpha >= 0.0) {
        const double al = ctx->opt.pc_alpha;
        k_gather<<<gz, 256, 0, s>>>(nnz, ctx->A_val, ctx->T_perm, ctx->T_val); CKL();
        k_row_abspow<<<gm, 256, 0, s>>>((int)m, ctx->A_rp, ctx->A_val, 2.0 - al, dr); CKL();
        k_row_abspow<<<gn, 256, 0, s>>>((int)n, ctx->T_rp, ctx->T_val, al, dc); CKL();
        k_factor<<<gm, 256, 0, s>>>((int)m, dr, ctx->Dr); CKL();
        k_factor<<<gn, 256, 0, s>>>((int)n, dc, ctx->Dc); CKL();
        k_scale_rows_cols<<<gm, 256, 0, s>>>((int)m, ctx->A_rp, ctx->A_ci, ctx->A_val, dr, dc); CKL();
    }
    k_gather<<<gz, 256, 0, s>>>(nnz, ctx->A_val, ctx->T_perm, ctx->T_val); CKL();

    const int gv = (int)((std::max(m, n) + TB - 1) / TB);
    k_prep_vectors<<<gv, TB, 0, s>>>((int)m, (int)n, ctx->Dr, ctx->Dc, ctx->b_s, ctx->c_s,
                                      ctx->l_s, ctx->u_s, ctx->partials, ctx->pstride);
    CKL();
    st = launch_reduce(ctx, {{Q_V2, gv}, {Q_V2B, gv}}, ctx->scal);
    if (st) return st;
    CK(cudaMemcpyAsync(ctx->scal_h, ctx->scal, sizeof(double) * NQ, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    ctx->beta_b = std::sqrt(ctx->scal_h[Q_V2]) + 1.0;
    ctx->beta_c = std::sqrt(ctx->scal_h[Q_V2B]) + 1.0;
    k_prep_normalise<<<grid_for(std::max(m, n)), 256, 0, s>>>((int)m, (int)n, ctx->beta_b, ctx->beta_c,
                                                              ctx->Dr, ctx->Dc, ctx->b_s, ctx->c_s,
                                                              ctx->l_s, ctx->u_s, ctx->wr, ctx->wc);
    CKL();
    // the iteration's copies: stored values through the position map, vectors renumbered
    k_gather_src<<<grid_for(ctx->SA.entries), 256, 0, s>>>(ctx->SA.entries, ctx->A_val, ctx->SA.src, ctx->SA.val); CKL();
    k_gather_src<<<grid_for(ctx->ST.entries), 256, 0, s>>>(ctx->ST.entries, ctx->T_val, ctx->ST.src, ctx->ST.val); CKL();
    k_narrow<<<grid_for(ctx->SA.entries), 256, 0, s>>>(ctx->SA.entries, ctx->SA.val, ctx->SA.val32); CKL();
    k_narrow<<<grid_for(ctx->ST.entries), 256, 0, s>>>(ctx->ST.entries, ctx->ST.val, ctx->ST.val32); CKL();
    k_permute<<<gm, 256, 0, s>>>(m, ctx->b_s, ctx->perm_r, ctx->bp); CKL();
    k_permute<<<gm, 256, 0, s>>>(m, ctx->wr, ctx->perm_r, ctx->wrp); CKL();
    k_permute<<<gn, 256, 0, s>>>(n, ctx->c_s, ctx->perm_c, ctx->cp); CKL();
    k_permute<<<gn, 256, 0, s>>>(n, ctx->l_s, ctx->perm_c, ctx->lp); CKL();
    k_permute<<<gn, 256, 0, s>>>(n, ctx->u_s, ctx->perm_c, ctx->up); CKL();
    k_permute<<<gn, 256, 0, s>>>(n, ctx->wc, ctx->perm_c, ctx->wcp); CKL();
    CK(cudaStreamSynchronize(s));
    if (ctx->opt.autotune) {
        int r1 = autotune_layout(ctx, false, rp, ci, pr, ipc);
        if (r1) return r1;
        r1 = autotune_layout(ctx, true, trp, tci, pc, ipr);
        if (r1) return r1;
    } else {
        const bool ra = smallA && op.sell_steps_a <= 0 && op.unit_cost_a <= 0.0;
        const bool rt = smallT && op.sell_steps_t <= 0 && op.unit_cost_t <= 0.0;
        if (ra || rt) {
            ctx->relayout.reset(new (std::nothrow) hpr_ctx::Relayout());
            if (!ctx->relayout) return fail_arg(ctx, HPR_ERR_NOMEM, "host copy of the layout structure");
            hpr_ctx::Relayout &R = *ctx->relayout;
            R.a = ra;
            R.t = rt;
            if (ra) { R.rp = std::move(rp); R.ci = std::move(ci); R.pr = std::move(pr); R.ipc = std::move(ipc); }
            if (rt) { R.trp = std::move(trp); R.tci = std::move(tci); R.pc = std::move(pc); R.ipr = std::move(ipr); }
        }
    }
    return HPR_OK;
}

// give a context's short-slice layouts (the small-phase rule) the default layout, for a
// batch whose fused phases move enough data to be bound by bandwidth, not by the longest
// unit's latency; captured graphs (they hold the old layouts' pointers) are dropped
int relayout_for_throughput(hpr_ctx *ctx, bool a, bool t)
{
    if (!ctx->relayout) return HPR_OK;
    hpr_ctx::Relayout &R = *ctx->relayout;
    a = a && R.a;
    t = t && R.t;
    if (!a && !t) return HPR_OK;
    int st;
    if (a) {
        SellHost H = build_sell(R.rp, R.ci, (int)ctx->m, R.pr, R.ipc, SELL_STEPS, UNIT_COST);
        if ((st = install_layout(ctx, ctx->SA, H, (int)ctx->m, ctx->A_val))) return st;
        R.a = false;
        R.rp.clear(); R.ci.clear(); R.pr.clear(); R.ipc.clear();
    }
    if (t) {
        SellHost H = build_sell(R.trp, R.tci, (int)ctx->n, R.pc, R.ipr, SELL_STEPS, UNIT_COST);
        if ((st = install_layout(ctx, ctx->ST, H, (int)ctx->n, ctx->T_val))) return st;
        R.t = false;
        R.trp.clear(); R.tci.clear(); R.pc.clear(); R.ipr.clear();
    }
    if (!R.a && !R.t) ctx->relayout.reset();
    for (auto &kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
    ctx->graphs.clear();
    if (ctx->pow_graph) cudaGraphExecDestroy(ctx->pow_graph);
    ctx->pow_graph = nullptr;
    const int need = std::max(ctx->SA.grid, ctx->ST.grid);   // one partial-sum slot per CTA
    if (need > ctx->pstride) {
        cudaFree(ctx->partials);
        ctx->partials = nullptr;
        ctx->pstride = need;
        DALLOC(ctx->partials, (int64_t)NQ * ctx->pstride);
    }
    return HPR_OK;
}

double merit_from(const double *S, double sigma, double lambda)
{
    // ||w - w_hat||_M = 2 ||w - w_bar||_M, eq. (def:M) with T1 = lambda I - A A^*
    const double q = sigma * lambda * S[Q_DY2] + 2.0 * S[Q_CROSS] + S[Q_DX2] / sigma;
    return 2.0 * std::sqrt(q > 0.0 ? q : 0.0);
}

}  // namespace

// ====================================================================== C ABI

extern "C" {

int hpr_default_options(hpr_options *o)
{
    if (!o) return HPR_ERR_ARG;
    memset(o, 0, sizeof *o);
    o->tol = 1e-8;
    o->max_iter = 10000000;
    o->time_limit_s = 0.0;
    o->check_every = 150;
    o->alpha1 = 0.2;
    o->alpha2 = 0.6;
    o->alpha3 = 0.2;
    o->sigma0 = 1.0;
    o->ruiz_iters = 10;
    o->pc_alpha = 1.0;
    o->power_max_iter = 5000;
    o->power_tol = 1e-10;
    o->seed = 0x48505221ULL;
    o->lambda_fixed = 0.0;
    o->restart = 1;
    o->sigma_update = 1;
    o->trace_iters = 0;
    o->use_graph = 1;
    o->verbose = 0;
    o->cuda_stream = nullptr;
    o->precision = 0;
    o->switch_tol = 1e-5;
    o->halpern = 1;
    o->reflect = 1;
    o->autotune = 0;
    o->sell_steps_a = o->sell_steps_t = 0;
    o->unit_cost_a = o->unit_cost_t = 0.0;
    o->sigma_policy = 0;
    o->policy_seed = 0x5167;
    o->policy_margin = 0.0;
    o->persistent = 1;
    o->pdl = 1;
    return HPR_OK;
}

static int check_options(hpr_ctx *ctx, const hpr_options *o)
{
    if (!(o->tol > 0.0)) return fail_arg(ctx, HPR_ERR_ARG, "tol must be > 0");
    if (o->max_iter < 1) return fail_arg(ctx, HPR_ERR_ARG, "max_iter must be >= 1");
    if (o->check_every < 1 || o->check_every > (1 << 20))
        return fail_arg(ctx, HPR_ERR_ARG, "check_every must be in [1, 2^20]");
    if (!(o->sigma0 > 0.0)) return fail_arg(ctx, HPR_ERR_ARG, "sigma0 must be > 0");
    if (o->ruiz_iters < 0) return fail_arg(ctx, HPR_ERR_ARG, "ruiz_iters must be >= 0");
    if (o->power_max_iter < 1) return fail_arg(ctx, HPR_ERR_ARG, "power_max_iter must be >= 1");
    if (o->trace_iters < 0) return fail_arg(ctx, HPR_ERR_ARG, "trace_iters must be >= 0");
    if (!(o->lambda_fixed >= 0.0)) return fail_arg(ctx, HPR_ERR_ARG, "lambda_fixed must be >= 0");
    if (o->precision != 0 && o->precision != 1) return fail_arg(ctx, HPR_ERR_ARG, "precision must be 0 or 1");
    if (!(o->switch_tol >= 0.0)) return fail_arg(ctx, HPR_ERR_ARG, "switch_tol must be >= 0");
    if (o->halpern != 0 && o->halpern != 1) return fail_arg(ctx, HPR_ERR_ARG, "halpern must be 0 or 1");
    if (o->reflect != 0 && o->reflect != 1) return fail_arg(ctx, HPR_ERR_ARG, "reflect must be 0 or 1");
    if (o->autotune != 0 && o->autotune != 1) return fail_arg(ctx, HPR_ERR_ARG, "autotune must be 0 or 1");
    if (o->sigma_policy < 0 || o->sigma_policy > 2) return fail_arg(ctx, HPR_ERR_ARG, "sigma_policy must be 0, 1 or 2");
    if (o->persistent < 0 || o->persistent > 2) return fail_arg(ctx, HPR_ERR_ARG, "persistent must be 0, 1 or 2");
    if (o->pdl != 0 && o->pdl != 1) return fail_arg(ctx, HPR_ERR_ARG, "pdl must be 0 or 1");
    if (!(o->policy_margin >= 0.0) || o->policy_margin > 100.0)
        return fail_arg(ctx, HPR_ERR_ARG, "policy_margin must be in [0, 100]");
    if (o->sell_steps_a < 0 || o->sell_steps_a > 4096 || o->sell_steps_t < 0 || o->sell_steps_t > 4096)
        return fail_arg(ctx, HPR_ERR_ARG, "sell_steps must be in [0, 4096]");
    if (!(o->unit_cost_a >= 0.0) || !(o->unit_cost_t >= 0.0) || o->unit_cost_a > 1e9 || o->unit_cost_t > 1e9)
        return fail_arg(ctx, HPR_ERR_ARG, "unit_cost must be in [0, 1e9]");
    return HPR_OK;
}

int hpr_create(hpr_ctx **out, const hpr_csr *A1, const hpr_csr *A2, const double *b1,
               const double *b2, const double *c, const double *l, const double *u,
               const hpr_options *opt)
{
    if (!out) return HPR_ERR_ARG;
    *out = nullptr;
    hpr_ctx *ctx = new (std::nothrow) hpr_ctx();
    if (!ctx) return HPR_ERR_NOMEM;
    auto bail = [&](int code) {
        g_static_err = "hpr_create failed (see hpr_last_error of a context)";
        static thread_local std::string last;
        last = ctx->err;
        g_static_err = last.c_str();
        free_all(ctx);
        delete ctx;
        return code;
    };
    if (opt) ctx->opt = *opt;
    else hpr_default_options(&ctx->opt);
    int st = check_options(ctx, &ctx->opt);
    if (st) return bail(st);

    int64_t r1 = 0, c1 = -1, r2 = 0, c2 = -1;
    if ((st = validate_block(ctx, A1, "A1", &r1, &c1))) return bail(st);
    if ((st = validate_block(ctx, A2, "A2", &r2, &c2))) return bail(st);
    int64_t n = c1 >= 0 ? c1 : c2;
    if (c1 >= 0 && c2 >= 0 && c1 != c2) return bail(fail_arg(ctx, HPR_ERR_ARG, "A1.cols != A2.cols"));
    if (n <= 0) return bail(fail_arg(ctx, HPR_ERR_ARG, "n must be >= 1"));
    const int64_t nnz = (r1 ? A1->nnz : 0) + (r2 ? A2->nnz : 0);
    if (r1 + r2 == 0 || nnz == 0) return bail(fail_arg(ctx, HPR_ERR_ZERO_MATRIX, "A has no nonzero entry"));
    if (nnz >= (int64_t)INT32_MAX || r1 + r2 >= (int64_t)INT32_MAX || n >= (int64_t)INT32_MAX)
        return bail(fail_arg(ctx, HPR_ERR_ARG, "sizes beyond 2^31-1 are not supported"));
    bool any_nonzero = false;
    for (int bI = 0; bI < 2 && !any_nonzero; ++bI) {
        const hpr_csr *B = bI ? A2 : A1;
        const int64_t rows = bI ? r2 : r1;
        if (!rows) continue;
        for (int64_t p = 0; p < B->nnz; ++p)
            if (B->val[p] != 0.0) { any_nonzero = true; break; }
    }
    if (!any_nonzero) return bail(fail_arg(ctx, HPR_ERR_ZERO_MATRIX, "A has no nonzero entry"));
    if ((r1 && !b1) || (r2 && !b2) || !c || !l || !u)
        return bail(fail_arg(ctx, HPR_ERR_ARG, "NULL vector"));
    for (int64_t i = 0; i < r1; ++i)
        if (!std::isfinite(b1[i])) return bail(fail_arg(ctx, HPR_ERR_ARG, "b1 not finite"));
    for (int64_t i = 0; i < r2; ++i)
        if (!std::isfinite(b2[i])) return bail(fail_arg(ctx, HPR_ERR_ARG, "b2 not finite"));
    for (int64_t j = 0; j < n; ++j) {
        if (!std::isfinite(c[j])) return bail(fail_arg(ctx, HPR_ERR_ARG, "c not finite"));
        if (std::isnan(l[j]) || std::isnan(u[j]) || l[j] > u[j] || l[j] == INFINITY || u[j] == -INFINITY)
            return bail(fail_arg(ctx, HPR_ERR_ARG, "bounds must satisfy l <= u, l < +inf, u > -inf"));
    }

    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) {
        ctx->err = "no CUDA device";
        (void)cudaGetLastError();
        return bail(HPR_ERR_NO_DEVICE);
    }
    cudaGetDevice(&ctx->device);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, ctx->device) != cudaSuccess || prop.major != 10 ||
        prop.minor != 3) {
        (void)cudaGetLastError();
        ctx->err = "this library is built for sm_103 (B300) only";
        return bail(HPR_ERR_NO_DEVICE);
    }
    ctx->num_sms = prop.multiProcessorCount;
    ctx->m1 = r1;
    ctx->m2 = r2;
    ctx->m = r1 + r2;
    ctx->n = n;
    ctx->nnz = nnz;
    {
        double sb = 0.0, sc = 0.0;
        for (int64_t i = 0; i < r1; ++i) sb += b1[i] * b1[i];
        for (int64_t i = 0; i < r2; ++i) sb += b2[i] * b2[i];
        for (int64_t j = 0; j < n; ++j) sc += c[j] * c[j];
        ctx->norm_b = std::sqrt(sb);
        ctx->norm_c = std::sqrt(sc);
    }
    if (ctx->opt.cuda_stream) {
        ctx->stream = (cudaStream_t)ctx->opt.cuda_stream;
    } else {
        e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bail(fail_cuda(ctx, e, "cudaStreamCreate", __LINE__));
        ctx->own_stream = true;
    }
    ctx->home_stream = ctx->stream;
    st = upload_and_prepare(ctx, A1, A2, b1, b2, c, l, u);
    if (st) return bail(st);
    *out = ctx;
    return HPR_OK;
}

int hpr_set_options(hpr_ctx *ctx, const hpr_options *opt)
{
    if (!ctx || !opt) return HPR_ERR_ARG;
    int st = check_options(ctx, opt);
    if (st) return st;
    void *old_stream = ctx->opt.cuda_stream;
    const int64_t ruiz = ctx->opt.ruiz_iters;
    const double pca = ctx->opt.pc_alpha;
    if (opt->seed != ctx->opt.seed || opt->power_tol != ctx->opt.power_tol ||
        opt->power_max_iter != ctx->opt.power_max_iter)
        ctx->have_power = false;
    if (opt->reflect != ctx->opt.reflect) {   // captured graphs hold the kernels' arguments
        for (auto &kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
        ctx->graphs.clear();
    }
    ctx->opt = *opt;
    ctx->opt.cuda_stream = old_stream;   // the stream is fixed at creation
    ctx->opt.ruiz_iters = ruiz;
    ctx->opt.pc_alpha = pca;
    return HPR_OK;
}

int hpr_power(hpr_ctx *ctx, double *lambda, int64_t *iters)
{
    if (!ctx) return HPR_ERR_ARG;
    cudaSetDevice(ctx->device);
    int st = run_power(ctx);
    if (st) return st;
    ctx->have_power = true;
    if (lambda) *lambda = ctx->lambda;
    if (iters) *iters = ctx->power_iters;
    return HPR_OK;
}

}  // extern "C"

namespace {

// ---------------------------------------------------------------- solve, in stages
// A solve is: solve_begin (power method, origin start), then periods of up to
// check_every iterations ending with a check -- period_prepare (control block of the
// period), the period's kernels, period_readback (check scalars to the host), one
// synchronisation, period_after (termination, restart and sigma decisions of the check)
// -- and solve_finish (back-map, summary).  hpr_solve runs one context through them;
// hpr_batch_solve runs many in lock step with fused kernels.

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the next output of the sequence at `state`
uint64_t splitmix64_next(uint64_t &state)
{
    uint64_t z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// The policy network's input at check record `rec`: the last 16 periodic checks up to and
// including it (the oldest repeated when fewer exist), each as log10 err_p, log10 err_d,
// log10 gap (floored at 1e-16) and log10 sigma, all divided by 8.
void policy_features(const std::vector<hpr_check_record> &recs, int64_t rec, float *out)
{
    std::vector<const hpr_check_record *> hist;
    for (int64_t i = rec; i >= 0 && hist.size() < 16; --i)
        if (recs[(size_t)i].kind & 1) hist.push_back(&recs[(size_t)i]);
    if (hist.empty()) hist.push_back(&recs[(size_t)rec]);
    while (hist.size() < 16) hist.push_back(hist.back());
    for (int j = 0; j < 16; ++j) {
        const hpr_check_record *c = hist[(size_t)(15 - j)];   // oldest first
        out[4 * j + 0] = (float)(std::log10(std::max(c->err_p, 1e-16)) / 8.0);
        out[4 * j + 1] = (float)(std::log10(std::max(c->err_d, 1e-16)) / 8.0);
        out[4 * j + 2] = (float)(std::log10(std::max(c->err_gap, 1e-16)) / 8.0);
        out[4 * j + 3] = (float)(std::log10(std::max(c->sigma, 1e-300)) / 8.0);
    }
}

// action of the policy network at the last check record: argmin of its five outputs
int policy_choose(hpr_ctx *ctx, int *action)
{
    float x[hprmlp::IN], q[hprmlp::OUT];
    policy_features(ctx->checks, (int64_t)ctx->checks.size() - 1, x);
    CK(cudaMemcpyAsync(ctx->policy_x, x, sizeof x, cudaMemcpyHostToDevice, ctx->stream));
    hprmlp::k_infer<<<1, hprmlp::TPB, 0, ctx->stream>>>(ctx->policy_wb, ctx->policy_x, 1, ctx->policy_q);
    CKL();
    ctx->launches += 1;
    CK(cudaMemcpyAsync(q, ctx->policy_q, sizeof q, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    int best = 0;
    for (int a = 1; a < hprmlp::OUT; ++a)
        if (q[a] < q[best]) best = a;
    if (!(q[best] < q[2] - ctx->opt.policy_margin)) best = 2;   // not clearly better: Algorithm 3's
    *action = best;
    return HPR_OK;
}

int solve_begin(hpr_ctx *ctx, double tol)
{
    hpr_options &o = ctx->opt;
    const int64_t n = ctx->n, m = ctx->m;
    cudaStream_t s = ctx->stream;
    ctx->solved = false;
    ctx->checks.clear();
    ctx->trace_written = 0;
    int st;

    // trace buffer
    if (o.trace_iters > 0) {
        const int64_t need = o.trace_iters;
        if (need != ctx->trace_n) {
            if (ctx->trace) cudaFree(ctx->trace);
            ctx->trace = nullptr;
            ctx->trace_n = 0;
            DALLOC(ctx->trace, need * (3 * n + 2 * m));
            ctx->trace_n = need;
        }
    }
    st = ensure_ctl(ctx, (int)std::min<int64_t>(o.check_every, o.max_iter));
    if (st) return st;

    CK(cudaStreamSynchronize(s));
    SolveState &S = ctx->ss;
    S = SolveState{};
    S.tol = tol;
    S.t0 = now_s();
    ctx->launches = 0;

    // ---- T1 = lambda I - A A^*: power method (counted in the solve time, Section 4.1)
    if (o.lambda_fixed > 0.0) {
        ctx->lambda = o.lambda_fixed;
        ctx->power_iters = 0;
        ctx->power_time = 0.0;
    } else {
        st = run_power(ctx);
        if (st) return st;
        ctx->power_time = now_s() - S.t0;
    }
    S.lambda = ctx->lambda;

    // ---- origin start, sigma_0 (Section 4.1)
    CK(cudaMemsetAsync(ctx->x, 0, sizeof(double) * n, s));
    CK(cudaMemsetAsync(ctx->x0, 0, sizeof(double) * n, s));
    CK(cudaMemsetAsync(ctx->y, 0, sizeof(double) * m, s));
    CK(cudaMemsetAsync(ctx->y0, 0, sizeof(double) * m, s));
    CK(cudaMemsetAsync(ctx->x32, 0, sizeof(float) * n, s));
    CK(cudaMemsetAsync(ctx->y32, 0, sizeof(float) * m, s));
    ctx->form = (int)o.precision;
    S.sigma = o.sigma0;
    S.status = HPR_MAX_ITER;
    S.tracing = ctx->trace_n > 0;
    S.done = o.max_iter <= 0;
    return HPR_OK;
}

// control block of the next period: sigma, 1/(lambda sigma) and the Halpern weights of
// its L iterations; fused_lo / fused_hi: the iterations that fused launches may run
int period_prepare(hpr_ctx *ctx, bool upload = true)
{
    SolveState &S = ctx->ss;
    const hpr_options &o = ctx->opt;
    const int64_t to_check = o.check_every - (S.k % o.check_every);
    S.L = (int)std::min<int64_t>(to_check, o.max_iter - S.k);
    S.first_r0 = (S.t == 0);
    DevCtl *h = ctx->ctl_h;
    h->sigma = S.sigma;
    h->inv_ls = 1.0 / (S.lambda * S.sigma);
    h->fused_lo = S.first_r0 ? 1 : 0;
    h->fused_hi = S.L - 1;
    h->form = ctx->form;
    h->active = S.done ? 0 : 1;
    h->check_a = S.first_r0 ? 0 : -1;
    h->check_b = S.L - 1;
    for (int i = 0; i < S.L; ++i) {
        const double tt = (double)(S.t + i);
        h->h[2 * i] = o.halpern ? 1.0 / (tt + 2.0) : 0.0;   // 0 and 1: w = w_target exactly
        h->h[2 * i + 1] = o.halpern ? (tt + 1.0) / (tt + 2.0) : 1.0;
    }
    if (upload)
        CK(cudaMemcpyAsync(ctx->ctl, h, sizeof(DevCtl) + sizeof(double) * 2 * S.L, cudaMemcpyHostToDevice,
                           ctx->stream));
    return HPR_OK;
}

// the period's kernels of a context run on its own (trace mode, a captured graph, or
// direct launches)
int period_enqueue_own(hpr_ctx *ctx)
{
    SolveState &S = ctx->ss;
    const hpr_options &o = ctx->opt;
    cudaStream_t s = ctx->stream;
    const int L = S.L;
    const bool first_r0 = S.first_r0;
    int st;
    const bool trace_period = S.tracing && S.k < ctx->trace_n;
    if (trace_period) {
        for (int i = 0; i < L; ++i) {
            const bool last = (i == L - 1);
            const bool r0 = (i == 0 && first_r0);
            // every traced iteration stores x_bar, y_bar; checks also reduce
            st = enqueue_iteration(ctx, i, true, last || r0, last ? 1 : 0);
            if (st) return st;
            if (!last) {
                st = trace_copy(ctx, S.k + i);
                if (st) return st;
            }
        }
    } else if (o.use_graph) {
        const GraphKey key{L, first_r0 ? 1 : 0, ctx->form};
        auto itg = ctx->graphs.find(key);
        if (itg == ctx->graphs.end()) {
            CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            const int64_t before = ctx->launches;
            int rr = enqueue_period(ctx, L, first_r0);
            ctx->graph_launches[key] = ctx->launches - before;
            ctx->launches = before;
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(s, &g);
            if (rr) { if (g) cudaGraphDestroy(g); return rr; }
            if (e != cudaSuccess) return fail_cuda(ctx, e, "cudaStreamEndCapture", __LINE__);
            cudaGraphExec_t ex = nullptr;
            e = cudaGraphInstantiate(&ex, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return fail_cuda(ctx, e, "cudaGraphInstantiate", __LINE__);
            itg = ctx->graphs.emplace(key, ex).first;
        }
        CK(cudaGraphLaunch(itg->second, s));
        ctx->launches += ctx->graph_launches[key];
    } else {
        st = enqueue_period(ctx, L, first_r0);
        if (st) return st;
    }
    return HPR_OK;
}

int period_readback(hpr_ctx *ctx)
{
    CK(cudaMemcpyAsync(ctx->scal_h, ctx->scal, sizeof(double) * 2 * NQ, cudaMemcpyDeviceToHost, ctx->stream));
    return HPR_OK;
}

// after the period's synchronisation: the check of its last iteration (termination test,
// restart criteria, SigmaUpdate, the FP32 -> FP64 switch) and the restart kernels
int period_after(hpr_ctx *ctx, double elapsed)
{
    SolveState &S = ctx->ss;
    const hpr_options &o = ctx->opt;
    const int64_t n = ctx->n, m = ctx->m;
    cudaStream_t s = ctx->stream;
    const double lambda = S.lambda;
    const int L = S.L;
    const bool first_r0 = S.first_r0;
    int st;

    const double *S1 = ctx->scal_h + NQ;
    const double *S0 = (first_r0 && L > 1) ? ctx->scal_h : S1;
    const int64_t kk = S.k + L - 1;           // index of the check iteration
    const int64_t tl = S.t + L - 1;           // its inner counter
    if (first_r0 && L > 1) {
        S.R0 = merit_from(S0, S.sigma, lambda);
        S.Rprev = S.R0;
        hpr_check_record rec{};
        rec.k = S.k; rec.r = S.r; rec.t = 0; rec.kind = 2; rec.cause = 0;
        rec.sigma = S.sigma; rec.Rt = S.R0; rec.R0 = S.R0; rec.sigma_next = S.sigma;
        rec.elapsed_s = elapsed; rec.action = -1; rec.sigma_rule = S.sigma;
        ctx->checks.push_back(rec);
    }
    const bool is_r0 = (tl == 0);
    const double Rt = merit_from(S1, S.sigma, lambda);
    if (is_r0) {
        S.R0 = Rt;
        S.Rprev = Rt;
    }
    // termination test of Section 4.1 in the original space
    const double bb = ctx->beta_b * ctx->beta_c;
    const double errp = std::sqrt(S1[Q_RP]) / (1.0 + ctx->norm_b);
    const double errd = std::sqrt(S1[Q_RD]) / (1.0 + ctx->norm_c);
    const double pobj = bb * S1[Q_CX];
    const double dobj = bb * (S1[Q_BY] + S1[Q_BND]);
    const double gap = std::fabs(dobj - pobj) / (1.0 + std::fabs(pobj) + std::fabs(dobj));
    const double kkt = std::max(errp, std::max(errd, gap));
    S.last_pobj = pobj; S.last_dobj = dobj; S.last_ep = errp; S.last_ed = errd; S.last_gap = gap; S.last_kkt = kkt;
    if (!std::isfinite(kkt) || !std::isfinite(Rt))
        return fail_arg(ctx, HPR_ERR_NUMERIC, "non-finite residual at iteration " + std::to_string(kk));
    if (S.time_1e4 < 0.0 && kkt <= 1e-4) {
        S.time_1e4 = elapsed;
        S.iters_1e4 = kk + 1;
    }

    int cause = 0;
    bool restart = false, stop = false;
    double sigma_next = S.sigma, Dx = 0.0, Dy = 0.0;
    if (kkt <= S.tol) {
        stop = true;
        S.status = HPR_OK;
        cause = -1;
    } else if (kk + 1 < o.max_iter && o.restart && !is_r0) {
        // restart criteria eq. (restart_1)-(restart_3)
        if (Rt <= o.alpha1 * S.R0) cause = 1;
        else if (Rt <= o.alpha2 * S.R0 && Rt > S.Rprev) cause = 2;
        else if ((double)(tl + 1) >= o.alpha3 * (double)(kk + 1)) cause = 3;
        S.Rprev = Rt;
        restart = cause != 0;
    }
    bool rule_sigma = false;                  // sigma_next is Delta_x / Delta_y
    if (restart) {
        // Algorithm 3 with eq. (sigma_T1!=0)
        Dx = std::sqrt(S1[Q_XX0]);
        Dy = std::sqrt(lambda) * std::sqrt(S1[Q_YY0]);
        const double ratio = errd / errp;
        rule_sigma = o.sigma_update && Dx > 1e-16 && Dx < 1e12 && Dy > 1e-16 && Dy < 1e12 &&
                     errp > 0.0 && ratio > 1e-8 && ratio < 1e8;
        if (rule_sigma)
            sigma_next = Dx / Dy;
        else
            sigma_next = o.sigma_update ? 1.0 : S.sigma;
    }
    // a learned sigma is watched until the next restart: a KKT residual above its value at
    // the decision sends the next restart back to Algorithm 3
    if (S.policy_watch && kkt > S.policy_kkt) {
        S.policy_suspend = true;
        S.policy_watch = false;
    }
    {
        hpr_check_record rec{};
        rec.k = kk; rec.r = S.r; rec.t = tl; rec.kind = 1 + (is_r0 ? 2 : 0); rec.cause = cause;
        rec.sigma = S.sigma; rec.err_p = errp; rec.err_d = errd; rec.err_gap = gap; rec.kkt = kkt;
        rec.pobj = pobj; rec.dobj = dobj; rec.Rt = Rt; rec.R0 = S.R0; rec.sigma_next = sigma_next;
        rec.Dx = Dx; rec.Dy = Dy; rec.elapsed_s = elapsed;
        rec.action = -1; rec.sigma_rule = sigma_next;
        ctx->checks.push_back(rec);
    }
    if (restart) S.policy_watch = false;      // a new inner loop: a new decision below
    if (restart && rule_sigma && o.sigma_policy != 0) {
        int action = -1;
        if (o.sigma_policy == 1) {
            uint64_t st64 = o.policy_seed ^ (0x9E3779B97F4A7C15ull * (uint64_t)(S.r + 1));
            action = (int)(splitmix64_next(st64) % (uint64_t)hprmlp::OUT);
        } else if (ctx->policy_wb) {
            if (S.policy_suspend) {
                S.policy_suspend = false;
                S.policy_fallbacks++;
            } else {
                if ((st = policy_choose(ctx, &action))) return st;
                S.policy_decisions++;
                S.policy_watch = true;
                S.policy_kkt = kkt;
            }
        }
        if (action >= 0) {
            sigma_next *= std::exp2(0.5 * (double)(action - 2));
            ctx->checks.back().action = action;
            ctx->checks.back().sigma_next = sigma_next;
        }
    }
    if (o.verbose)
        fprintf(stderr, "hpr k=%lld r=%lld t=%lld sigma=%.3e kkt=%.3e (p %.2e d %.2e g %.2e) R=%.3e cause=%d %.3fs\n",
                (long long)(kk + 1), (long long)S.r, (long long)tl, S.sigma, kkt, errp, errd, gap, Rt,
                cause, elapsed);

    if (ctx->form == 1) S.iters_fp32 = kk + 1;
    // the FP32 form hands over to FP64 iterates at the first check below switch_tol
    const bool widen = ctx->form == 1 && !stop && kkt < o.switch_tol;
    if (widen) ctx->form = 0;
    if (restart && ctx->form == 1) {
        k_restart32<<<grid_for(n + m), 256, 0, s>>>((int)n, (int)m, ctx->xbar, ctx->ybar, ctx->x32,
                                                    ctx->x0, ctx->y32, ctx->y0);
        CKL();
        ctx->launches += 1;
    } else if (restart) {
        k_restart<<<grid_for(n + m), 256, 0, s>>>((int)n, (int)m, ctx->xbar, ctx->ybar, ctx->x,
                                                  ctx->x0, ctx->y, ctx->y0);
        CKL();
        ctx->launches += 1;
    } else if (widen) {
        k_widen<<<grid_for(n + m), 256, 0, s>>>((int)n, (int)m, ctx->x32, ctx->y32, ctx->x, ctx->y);
        CKL();
        ctx->launches += 1;
    }
    if (restart) {
        S.sigma = sigma_next;
        S.t = 0;
        S.r++;
    } else {
        S.t = tl + 1;
    }
    if (S.tracing && kk < ctx->trace_n) {
        st = trace_copy(ctx, kk);
        if (st) return st;
    }
    S.k = kk + 1;
    if (stop) {
        S.done = true;
    } else if (o.time_limit_s > 0.0 && elapsed >= o.time_limit_s && S.k < o.max_iter) {
        S.status = HPR_TIME_LIMIT;
        S.done = true;
    } else if (S.k >= o.max_iter) {
        S.done = true;
    }
    return HPR_OK;
}

// output: the last w_bar mapped back to the original LP, and the summary
int solve_finish(hpr_ctx *ctx)
{
    SolveState &S = ctx->ss;
    const int64_t n = ctx->n, m = ctx->m;
    cudaStream_t s = ctx->stream;
    k_backmap<<<grid_for(n + m), 256, 0, s>>>((int)n, (int)m, ctx->beta_b, ctx->beta_c, ctx->xbar,
                                              ctx->ybar, ctx->zbar, ctx->perm_c, ctx->perm_r, ctx->Dr,
                                              ctx->Dc, ctx->l_o, ctx->u_o, ctx->xo, ctx->yo, ctx->zo);
    CKL();
    ctx->launches += 1;
    CK(cudaStreamSynchronize(s));
    const double total = now_s() - S.t0;

    hpr_info &I = ctx->info;
    memset(&I, 0, sizeof I);
    I.primal_obj = S.last_pobj; I.dual_obj = S.last_dobj; I.err_p = S.last_ep; I.err_d = S.last_ed;
    I.err_gap = S.last_gap; I.kkt = S.last_kkt; I.sigma = S.sigma; I.lambda = S.lambda;
    I.solve_time_s = total; I.power_time_s = ctx->power_time;
    I.time_to_1e4_s = S.time_1e4; I.iters_to_1e4 = S.iters_1e4;
    I.iters = S.k; I.restarts = S.r; I.power_iters = ctx->power_iters;
    I.n_checks = (int64_t)ctx->checks.size(); I.launches = ctx->launches; I.status = S.status;
    I.iters_fp32 = S.iters_fp32;
    I.policy_decisions = S.policy_decisions;
    I.policy_fallbacks = S.policy_fallbacks;
    ctx->solved = true;
    return S.status;
}

constexpr size_t SMALL_SMEM_MAX = 200 * 1024;
// One SM issues the FP64 work of the whole iteration: about one warp instruction per 32
// stored entries of A and A^T plus ~8 per 32-row slice (row sums' tails and epilogues), at
// ~17 cycles each.  Measured on the tiny planted LP, QAPs (N = 5, 6) and medium planted LPs
// at 1/1000 .. 1/200 scale, an iteration of the single CTA costs ~1.5 us + 8.4 ns per such
// instruction, and the multi-CTA graph path ~5 us (launch-bound) or more; the default takes
// the single CTA up to 600 instructions (~6.5 us).
constexpr double SMALL_FP64_MAX = 600.0;

double small_fp64_per_iter(const hpr_ctx *ctx)
{
    return (double)(ctx->SA.entries + ctx->ST.entries) / 32.0 + 8.0 * (double)(ctx->SA.nslices + ctx->ST.nslices);
}

// whether the persistent single-CTA path can run this solve (and why not); unless forced,
// also whether it is expected to be the faster path
const char *small_unfit(const hpr_ctx *ctx, bool forced)
{
    const hpr_options &o = ctx->opt;
    if (hprsmall::small_vec_bytes((int)ctx->m, (int)ctx->n) > SMALL_SMEM_MAX)
        return "the iterates do not fit in shared memory";
    if (o.precision != 0) return "the FP32 form";
    if (o.trace_iters > 0) return "tracing";
    if (o.time_limit_s > 0.0) return "a time limit";
    if (o.sigma_policy != 0) return "a sigma policy";
    if (!forced && small_fp64_per_iter(ctx) > SMALL_FP64_MAX) return "more FP64 work per iteration than one SM takes faster";
    return nullptr;
}

// the launch arguments of a single-CTA solve of ctx with tolerance tol, and its dynamic
// shared memory; resets the context's solve state (buffers for the check records and the
// results are allocated on first use and kept)
int small_prepare(hpr_ctx *ctx, double tol, hprsmall::SmallArgs &A, size_t *smem)
{
    using namespace hprsmall;
    const hpr_options &o = ctx->opt;
    const int64_t n = ctx->n, m = ctx->m;
    cudaStream_t s = ctx->stream;
    ctx->solved = false;
    ctx->checks.clear();
    ctx->trace_written = 0;
    CK(cudaStreamSynchronize(s));
    SolveState &S = ctx->ss;
    S = SolveState{};
    S.tol = tol;
    S.t0 = now_s();
    ctx->launches = 0;
    const int cap = (int)std::min<int64_t>(1 << 16, 2 * (o.max_iter / o.check_every) + 16);
    if (cap > ctx->small_cap) {                // kept between solves
        if (ctx->small_recs) cudaFree(ctx->small_recs);
        ctx->small_recs = nullptr;
        ctx->small_cap = 0;
        DALLOC(ctx->small_recs, cap);
        ctx->small_cap = cap;
    }
    if (!ctx->small_out) DALLOC(ctx->small_out, SO_LEN);
    auto mat_of = [](const SellDev &D) {
        SmallMat M{};
        M.nslices = D.nslices; M.entries = D.entries;
        M.srow = D.srow; M.sptr = D.sptr; M.col = D.col; M.slg = D.slg; M.val = D.val;
        return M;
    };
    A = SmallArgs{};
    A.m = (int)m; A.n = (int)n;
    A.A = mat_of(ctx->SA); A.T = mat_of(ctx->ST);
    A.ineq = ctx->ineq;
    A.b = ctx->bp; A.c = ctx->cp; A.l = ctx->lp; A.u = ctx->up; A.wr = ctx->wrp; A.wc = ctx->wcp;
    A.beta_b = ctx->beta_b; A.beta_c = ctx->beta_c; A.norm_b = ctx->norm_b; A.norm_c = ctx->norm_c;
    A.tol = tol; A.alpha1 = o.alpha1; A.alpha2 = o.alpha2; A.alpha3 = o.alpha3; A.sigma0 = o.sigma0;
    A.lambda_fixed = o.lambda_fixed; A.power_tol = o.power_tol;
    A.max_iter = o.max_iter; A.check_every = o.check_every; A.power_max_iter = std::max<int64_t>(1, o.power_max_iter);
    A.seed = o.seed;
    A.restart = (int)o.restart; A.sigma_update = (int)o.sigma_update; A.halpern = (int)o.halpern;
    A.reflect = (int)o.reflect;
    A.mat_smem = small_smem_bytes((int)m, (int)n, A.A, A.T, true) <= SMALL_SMEM_MAX ? 1 : 0;
    A.perm_r = ctx->perm_r;
    A.xbar_out = ctx->xbar; A.ybar_out = ctx->ybar; A.zbar_out = ctx->zbar;
    A.recs = ctx->small_recs; A.rec_cap = cap; A.out = ctx->small_out;
    *smem = small_smem_bytes((int)m, (int)n, A.A, A.T, A.mat_smem != 0);
    return HPR_OK;
}

// a finished single-CTA solve into the context's state: its results, check records and
// the back-map to the original LP
int small_collect(hpr_ctx *ctx)
{
    using namespace hprsmall;
    SolveState &S = ctx->ss;
    double h[SO_LEN];
    cudaError_t e = cudaMemcpyAsync(h, ctx->small_out, sizeof h, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return fail_cuda(ctx, e, "solve_small", __LINE__);
    ctx->launches = 1;
    const int64_t nrec = std::min<int64_t>((int64_t)h[SO_NREC], ctx->small_cap);
    ctx->checks.resize((size_t)nrec);
    if (nrec && cudaMemcpy(ctx->checks.data(), ctx->small_recs, sizeof(hpr_check_record) * nrec,
                           cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail_arg(ctx, HPR_ERR_CUDA, "solve_small: check records");
    ctx->lambda = h[SO_LAMBDA];
    ctx->power_iters = (int64_t)h[SO_POWER_ITERS];
    ctx->power_time = h[SO_POWER_S];
    S.lambda = h[SO_LAMBDA];
    S.k = (int64_t)h[SO_ITERS]; S.r = (int64_t)h[SO_RESTARTS]; S.sigma = h[SO_SIGMA];
    S.status = (int)h[SO_STATUS];
    S.last_pobj = h[SO_POBJ]; S.last_dobj = h[SO_DOBJ]; S.last_ep = h[SO_ERRP]; S.last_ed = h[SO_ERRD];
    S.last_gap = h[SO_GAP]; S.last_kkt = h[SO_KKT];
    S.time_1e4 = h[SO_T1E4] >= 0.0 ? h[SO_T1E4] : -1.0;
    S.iters_1e4 = (int64_t)h[SO_I1E4];
    S.done = true;
    if (S.status == HPR_ERR_NUMERIC)
        return fail_arg(ctx, HPR_ERR_NUMERIC, "non-finite residual at iteration " + std::to_string(S.k - 1));
    return solve_finish(ctx);
}

// launches k_solve_small over `count` argument blocks (one CTA each) on stream s
cudaError_t small_launch(const hprsmall::SmallArgs *args_dev, int count, size_t smem, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(hprsmall::k_solve_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    hprsmall::k_solve_small<<<count, hprsmall::NT, smem, s>>>(args_dev);
    return cudaGetLastError();
}

int solve_small(hpr_ctx *ctx, double tol)
{
    using namespace hprsmall;
    SmallArgs A;
    size_t smem = 0;
    int st = small_prepare(ctx, tol, A, &smem);
    if (st) return st;
    if (!ctx->small_args) DALLOC(ctx->small_args, 1);
    cudaError_t e = cudaMemcpyAsync(ctx->small_args, &A, sizeof A, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = small_launch(ctx->small_args, 1, smem, ctx->stream);
    if (e != cudaSuccess) return fail_cuda(ctx, e, "solve_small", __LINE__);
    return small_collect(ctx);
}

}  // namespace

extern "C" {

int hpr_solve(hpr_ctx *ctx, double tol)
{
    if (!ctx) return HPR_ERR_ARG;
    if (!(tol > 0.0)) return fail_arg(ctx, HPR_ERR_ARG, "tol must be > 0");
    if (ctx->batched) return fail_arg(ctx, HPR_ERR_STATE, "the context belongs to a batch");
    cudaSetDevice(ctx->device);
    if (ctx->opt.persistent) {
        const char *why = small_unfit(ctx, ctx->opt.persistent == 2);
        if (!why) return solve_small(ctx, tol);
        if (ctx->opt.persistent == 2)
            return fail_arg(ctx, HPR_ERR_ARG, std::string("persistent = 2 but the single-CTA path cannot run: ") + why);
    }
    int st = solve_begin(ctx, tol);
    if (st) return st;
    SolveState &S = ctx->ss;
    while (!S.done) {
        if ((st = period_prepare(ctx))) return st;
        if ((st = period_enqueue_own(ctx))) return st;
        if ((st = period_readback(ctx))) return st;
        CK(cudaStreamSynchronize(ctx->stream));
        if ((st = period_after(ctx, now_s() - S.t0))) return st;
    }
    return solve_finish(ctx);
}

int hpr_get(const hpr_ctx *cctx, double *x, double *y, double *z, hpr_info *info)
{
    if (!cctx) return HPR_ERR_ARG;
    hpr_ctx *ctx = const_cast<hpr_ctx *>(cctx);
    if (!ctx->solved) return fail_arg(ctx, HPR_ERR_STATE, "no solve has completed");
    cudaSetDevice(ctx->device);
    if (x) CK(cudaMemcpyAsync(x, ctx->xo, sizeof(double) * ctx->n, cudaMemcpyDeviceToHost, ctx->stream));
    if (y) CK(cudaMemcpyAsync(y, ctx->yo, sizeof(double) * ctx->m, cudaMemcpyDeviceToHost, ctx->stream));
    if (z) CK(cudaMemcpyAsync(z, ctx->zo, sizeof(double) * ctx->n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (info) *info = ctx->info;
    return HPR_OK;
}

int hpr_get_scaling(const hpr_ctx *cctx, double *Dr, double *Dc, double *As_val, double *bs,
                    double *cs, double *ls, double *us, double *beta)
{
    if (!cctx) return HPR_ERR_ARG;
    hpr_ctx *ctx = const_cast<hpr_ctx *>(cctx);
    cudaSetDevice(ctx->device);
    cudaStream_t s = ctx->stream;
    if (Dr) CK(cudaMemcpyAsync(Dr, ctx->Dr, sizeof(double) * ctx->m, cudaMemcpyDeviceToHost, s));
    if (Dc) CK(cudaMemcpyAsync(Dc, ctx->Dc, sizeof(double) * ctx->n, cudaMemcpyDeviceToHost, s));
    if (As_val) CK(cudaMemcpyAsync(As_val, ctx->A_val, sizeof(double) * ctx->nnz, cudaMemcpyDeviceToHost, s));
    if (bs) CK(cudaMemcpyAsync(bs, ctx->b_s, sizeof(double) * ctx->m, cudaMemcpyDeviceToHost, s));
    if (cs) CK(cudaMemcpyAsync(cs, ctx->c_s, sizeof(double) * ctx->n, cudaMemcpyDeviceToHost, s));
    if (ls) CK(cudaMemcpyAsync(ls, ctx->l_s, sizeof(double) * ctx->n, cudaMemcpyDeviceToHost, s));
    if (us) CK(cudaMemcpyAsync(us, ctx->u_s, sizeof(double) * ctx->n, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (beta) {
        beta[0] = ctx->beta_b;
        beta[1] = ctx->beta_c;
    }
    return HPR_OK;
}

int hpr_get_layout(const hpr_ctx *ctx, int64_t *sell_steps, double *unit_cost, int64_t *units)
{
    if (!ctx) return HPR_ERR_ARG;
    if (sell_steps) { sell_steps[0] = ctx->SA.steps_max; sell_steps[1] = ctx->ST.steps_max; }
    if (unit_cost) { unit_cost[0] = ctx->SA.unit_cost; unit_cost[1] = ctx->ST.unit_cost; }
    if (units) { units[0] = ctx->SA.nruns; units[1] = ctx->ST.nruns; }
    return HPR_OK;
}

int hpr_layout_plan(const hpr_csr *B, int64_t steps_max, double unit_cost, int64_t *nslices, int64_t *entries,
                    int64_t *units, int32_t *row_order, int32_t *srow, int32_t *sptr, uint8_t *slg, int32_t *col,
                    int32_t *src, int32_t *wstart)
{
    if (!B || B->rows < 0 || B->cols < 0 || B->nnz < 0 || B->rows >= (int64_t)INT32_MAX ||
        B->cols >= (int64_t)INT32_MAX || B->nnz >= (int64_t)INT32_MAX || !B->row_ptr ||
        (B->nnz > 0 && !B->col_idx) || !(steps_max >= 1 && steps_max <= 4096) || !(unit_cost > 0.0)) {
        g_static_err = "hpr_layout_plan: bad matrix or parameters";
        return HPR_ERR_ARG;
    }
    const int rows = (int)B->rows;
    if (B->row_ptr[0] != 0 || B->row_ptr[rows] != B->nnz) {
        g_static_err = "hpr_layout_plan: row_ptr[0] != 0 or row_ptr[rows] != nnz";
        return HPR_ERR_ARG;
    }
    std::vector<int> rp((size_t)rows + 1), ci((size_t)std::max<int64_t>(B->nnz, 1), 0), icol((size_t)B->cols);
    for (int i = 0; i <= rows; ++i) {
        rp[(size_t)i] = (int)B->row_ptr[i];
        if (i > 0 && rp[(size_t)i] < rp[(size_t)i - 1]) {
            g_static_err = "hpr_layout_plan: row_ptr decreases";
            return HPR_ERR_ARG;
        }
    }
    for (int64_t p = 0; p < B->nnz; ++p) {
        if (B->col_idx[p] < 0 || B->col_idx[p] >= B->cols) {
            g_static_err = "hpr_layout_plan: column index out of range";
            return HPR_ERR_ARG;
        }
        ci[(size_t)p] = B->col_idx[p];
    }
    for (int64_t j = 0; j < B->cols; ++j) icol[(size_t)j] = (int)j;
    const std::vector<int> perm = order_by_length(rp, rows);
    const SellHost H = build_sell(rp, ci, rows, perm, icol, (int)steps_max, unit_cost);
    const int64_t nu = (int64_t)H.wstart.size() - 1;
    if (nslices) *nslices = H.nslices;
    if (entries) *entries = (int64_t)H.col.size();
    if (units) *units = nu;
    auto put = [](int32_t *dst, const std::vector<int> &v) {
        if (dst && !v.empty()) memcpy(dst, v.data(), sizeof(int32_t) * v.size());
    };
    put(row_order, perm);
    put(srow, H.srow);
    put(sptr, H.sptr);
    put(col, H.col);
    put(src, H.src);
    put(wstart, H.wstart);
    if (slg && !H.slg.empty()) memcpy(slg, H.slg.data(), H.slg.size());
    return HPR_OK;
}

int hpr_get_checks(const hpr_ctx *ctx, hpr_check_record *out, int64_t cap, int64_t *count)
{
    if (!ctx) return HPR_ERR_ARG;
    const int64_t cnt = (int64_t)ctx->checks.size();
    if (count) *count = cnt;
    if (out && cap > 0) memcpy(out, ctx->checks.data(), sizeof(hpr_check_record) * (size_t)std::min(cap, cnt));
    return HPR_OK;
}

int hpr_get_trace(const hpr_ctx *cctx, int64_t k, double *xbar, double *xhat, double *x,
                  double *ybar, double *y)
{
    if (!cctx) return HPR_ERR_ARG;
    hpr_ctx *ctx = const_cast<hpr_ctx *>(cctx);
    if (k < 0 || k >= ctx->trace_written) return fail_arg(ctx, HPR_ERR_STATE, "iteration not traced");
    cudaSetDevice(ctx->device);
    const int64_t n = ctx->n, m = ctx->m;
    const double *rec = ctx->trace + (size_t)k * (size_t)(3 * n + 2 * m);
    cudaStream_t s = ctx->stream;
    // the trace holds renumbered vectors: restore the original order on the way out
    double *outs[5] = {xbar, xhat, x, ybar, y};
    const int64_t off[5] = {0, n, 2 * n, 3 * n, 3 * n + m};
    for (int v = 0; v < 5; ++v) {
        if (!outs[v]) continue;
        const bool isx = v < 3;
        const int64_t len = isx ? n : m;
        k_unpermute<<<grid_for(len), 256, 0, s>>>(len, rec + off[v], isx ? ctx->perm_c : ctx->perm_r, ctx->unperm);
        CKL();
        CK(cudaMemcpyAsync(outs[v], ctx->unperm, sizeof(double) * len, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return HPR_OK;
}

int hpr_time_iteration(hpr_ctx *ctx, int64_t reps, double *ms_x, double *ms_y, double *ms_iter)
{
    if (!ctx || reps < 1) return HPR_ERR_ARG;
    if (!ctx->solved) return fail_arg(ctx, HPR_ERR_STATE, "no solve has completed");
    cudaSetDevice(ctx->device);
    cudaStream_t s = ctx->stream;
    // coefficients of a mid-run Halpern step; the timing does not depend on them
    DevCtl *h = ctx->ctl_h;
    h->sigma = ctx->info.sigma > 0.0 ? ctx->info.sigma : 1.0;
    h->inv_ls = 1.0 / (ctx->lambda * h->sigma);
    h->h[0] = 1.0 / 1002.0;
    h->h[1] = 1001.0 / 1002.0;
    CK(cudaMemcpyAsync(ctx->ctl, h, sizeof(DevCtl), cudaMemcpyHostToDevice, s));
    // reps back-to-back iterations (phase X, phase Y) with events between the phases and no
    // host synchronisation in between, so the launch queue stays ahead of the GPU; the first
    // two iterations are left out of the averages (the queue fills during them)
    const int64_t warm = 2, total = reps + warm;
    std::vector<cudaEvent_t> ev((size_t)(2 * total + 1), nullptr);
    int rc = HPR_OK;
    for (auto &e : ev) {
        cudaError_t ce = cudaEventCreate(&e);
        if (ce != cudaSuccess) { e = nullptr; rc = fail_cuda(ctx, ce, "hpr_time_iteration", __LINE__); break; }
    }
    const bool f32 = ctx->opt.precision == 1;
    if (rc == HPR_OK) rc = (cudaEventRecord(ev[0], s) == cudaSuccess) ? HPR_OK : HPR_ERR_CUDA;
    for (int64_t r = 0; r < total && rc == HPR_OK; ++r) {
        rc = f32 ? launch_sell(ctx, ctx->ST, epi_x32<false>(ctx, 0))
                 : launch_sell(ctx, ctx->ST, epi_x<false>(ctx, 0));
        if (rc) break;
        cudaEventRecord(ev[(size_t)(2 * r + 1)], s);
        rc = f32 ? launch_sell(ctx, ctx->SA, epi_y32<false>(ctx, 0))
                 : launch_sell(ctx, ctx->SA, epi_y<false>(ctx, 0));
        if (rc) break;
        cudaEventRecord(ev[(size_t)(2 * r + 2)], s);
    }
    double tx = 0.0, ty = 0.0;
    if (rc == HPR_OK) {
        cudaError_t e = cudaEventSynchronize(ev.back());
        if (e != cudaSuccess) rc = fail_cuda(ctx, e, "hpr_time_iteration", __LINE__);
    }
    for (int64_t r = warm; r < total && rc == HPR_OK; ++r) {
        float a = 0.f, b = 0.f;
        cudaEventElapsedTime(&a, ev[(size_t)(2 * r)], ev[(size_t)(2 * r + 1)]);
        cudaEventElapsedTime(&b, ev[(size_t)(2 * r + 1)], ev[(size_t)(2 * r + 2)]);
        tx += a;
        ty += b;
    }
    for (auto &e : ev)
        if (e) cudaEventDestroy(e);
    if (rc) return rc;
    if (ms_x) *ms_x = tx / (double)reps;
    if (ms_y) *ms_y = ty / (double)reps;
    if (ms_iter) *ms_iter = (tx + ty) / (double)reps;
    return HPR_OK;
}

const char *hpr_last_error(const hpr_ctx *ctx)
{
    return ctx ? ctx->err.c_str() : g_static_err;
}

const char *hpr_status_str(int s)
{
    switch (s) {
    case HPR_OK: return "HPR_OK";
    case HPR_MAX_ITER: return "HPR_MAX_ITER";
    case HPR_TIME_LIMIT: return "HPR_TIME_LIMIT";
    case HPR_ERR_ARG: return "HPR_ERR_ARG";
    case HPR_ERR_ZERO_MATRIX: return "HPR_ERR_ZERO_MATRIX";
    case HPR_ERR_NOMEM: return "HPR_ERR_NOMEM";
    case HPR_ERR_CUDA: return "HPR_ERR_CUDA";
    case HPR_ERR_DEVICE_TIMEOUT: return "HPR_ERR_DEVICE_TIMEOUT";
    case HPR_ERR_NUMERIC: return "HPR_ERR_NUMERIC";
    case HPR_ERR_STATE: return "HPR_ERR_STATE";
    case HPR_ERR_NO_DEVICE: return "HPR_ERR_NO_DEVICE";
    default: return "HPR_UNKNOWN";
    }
}

void hpr_destroy(hpr_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    ctx->stream = ctx->home_stream;
    free_all(ctx);
    delete ctx;
}

}  // extern "C"

// ====================================================================== batched solve
// Many LPs, one context each, solved in lock step: every period, the normal iterations of
// all contexts run as fused launches over one work list (k_sell_multi, captured as a CUDA
// graph per period length and set of forms), while each context's check iterations,
// residual passes and reductions, and its decisions, stay its own.  Contexts that have
// converged drop out of the fused launches through their control blocks.

struct hpr_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<hpr_ctx *> ctxs;
    MultiTask *tasksT = nullptr, *tasksA = nullptr;   // fused CTA lists (A^T and A phases)
    int ntasksT = 0, ntasksA = 0;
    SellArgs *sellT64 = nullptr, *sellA64 = nullptr, *sellT32 = nullptr, *sellA32 = nullptr;
    EpiX<false> *ex = nullptr;
    EpiY<false> *ey = nullptr;
    EpiX32<false> *ex32 = nullptr;
    EpiY32<false> *ey32 = nullptr;
    EpiX<true> *exc = nullptr;
    EpiY<true> *eyc = nullptr;
    EpiX32<true> *exc32 = nullptr;
    EpiY32<true> *eyc32 = nullptr;
    EpiDual *edual = nullptr;
    EpiPrimal *eprim = nullptr;
    RedTask *red = nullptr;
    int nred = 0;
    // every context's control block and check scalars in one array each (one copy a period)
    char *ctl_all = nullptr, *ctl_all_h = nullptr;
    size_t ctl_stride = 0, ctl_cap_bytes = 0;
    double *scal_all = nullptr, *scal_all_h = nullptr;
    std::map<std::pair<int, int>, cudaGraphExec_t> graphs;   // (L, forms present)
    std::map<std::pair<int, int>, int64_t> graph_nodes;      // kernels in each
    int64_t power_threads = 8;
    double solve_time = 0.0;
    int64_t periods = 0, fused_launches = 0;
    hprsmall::SmallArgs *small_args = nullptr;   // single-CTA launch: one argument block per LP
    size_t small_cap = 0;
};

namespace {

void batch_free(hpr_batch *b)
{
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
    void *dev[] = {b->tasksT, b->tasksA, b->sellT64, b->sellA64, b->sellT32, b->sellA32, b->ex, b->ey,
                   b->ex32, b->ey32, b->exc, b->eyc, b->exc32, b->eyc32, b->edual, b->eprim, b->red,
                   b->ctl_all, b->scal_all, b->small_args};
    for (void *p : dev)
        if (p) cudaFree(p);
    if (b->ctl_all_h) cudaFreeHost(b->ctl_all_h);
    if (b->scal_all_h) cudaFreeHost(b->scal_all_h);
    for (hpr_ctx *c : b->ctxs) {
        c->stream = c->home_stream;
        c->batched = false;
    }
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
}

// whether every context of the batch would take the persistent single-CTA path on its own
bool batch_all_small(const hpr_batch *b)
{
    for (const hpr_ctx *c : b->ctxs)
        if (c->opt.persistent == 0 || small_unfit(c, c->opt.persistent == 2)) return false;
    return true;
}

// A batch of LPs that all take the persistent single-CTA path: one launch of k_solve_small
// with one CTA per LP (each LP on an SM of its own, the LPs independent of one another), then
// each context's results read back as after its own solve.
int batch_small(hpr_batch *b, double tol)
{
    using namespace hprsmall;
    std::vector<hpr_ctx *> &cs = b->ctxs;
    const double t0 = now_s();
    std::vector<SmallArgs> args(cs.size());
    size_t smem = 0;
    for (size_t i = 0; i < cs.size(); ++i) {
        size_t si = 0;
        const int st = small_prepare(cs[i], tol, args[i], &si);
        if (st) return st;
        smem = std::max(smem, si);
    }
    if (b->small_cap < cs.size()) {
        if (b->small_args) cudaFree(b->small_args);
        b->small_args = nullptr;
        b->small_cap = 0;
        if (cudaMalloc((void **)&b->small_args, sizeof(SmallArgs) * cs.size()) != cudaSuccess) {
            g_static_err = "hpr_batch_solve: single-CTA arguments could not be allocated";
            return HPR_ERR_NOMEM;
        }
        b->small_cap = cs.size();
    }
    cudaError_t e = cudaMemcpyAsync(b->small_args, args.data(), sizeof(SmallArgs) * cs.size(),
                                    cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = small_launch(b->small_args, (int)cs.size(), smem, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        g_static_err = "hpr_batch_solve: single-CTA launch failed";
        return HPR_ERR_CUDA;
    }
    int status = HPR_OK;
    for (hpr_ctx *c : cs) {
        const int st = small_collect(c);
        if (st < 0) return st;
        if (st != HPR_OK && status == HPR_OK) status = st;
    }
    b->periods = 0;
    b->fused_launches = 1;
    b->solve_time = now_s() - t0;
    return status;
}

template <class T>
int upload_table(const std::vector<T> &h, T **d)
{
    if (cudaMalloc((void **)d, sizeof(T) * std::max<size_t>(1, h.size())) != cudaSuccess) return HPR_ERR_NOMEM;
    if (!h.empty() && cudaMemcpy(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return HPR_ERR_CUDA;
    return HPR_OK;
}

// fused CTA list of one phase: every CTA of every context's own launch, costliest first
// (cost: its SELL_WARPS work units), ties by context and CTA
std::vector<MultiTask> fused_tasks(const std::vector<hpr_ctx *> &cs, bool transpose)
{
    struct T { float cost; int inst, cta; };
    std::vector<T> all;
    for (size_t i = 0; i < cs.size(); ++i) {
        const SellDev &M = transpose ? cs[i]->ST : cs[i]->SA;
        if (M.rows == 0) continue;
        for (int c = 0; c < M.grid; ++c) {
            float cost = 0.f;
            for (int r = c * SELL_WARPS; r < std::min(M.nruns, (c + 1) * SELL_WARPS); ++r) cost += M.ucost[(size_t)r];
            all.push_back({cost, (int)i, c});
        }
    }
    std::stable_sort(all.begin(), all.end(), [](const T &a, const T &b) { return a.cost > b.cost; });
    std::vector<MultiTask> out(all.size());
    for (size_t i = 0; i < all.size(); ++i) out[i] = MultiTask{all[i].inst, all[i].cta};
    return out;
}

// per-context layouts, epilogue operands and reduction tasks of the fused launches
// (allocated once, refreshed before every solve: a solve may reallocate a context's
// control block, and a batched solve points it into the batch's array)
int batch_tables(hpr_batch *b, bool alloc)
{
    std::vector<SellArgs> sT64, sA64, sT32, sA32;
    std::vector<EpiX<false>> ex;
    std::vector<EpiY<false>> ey;
    std::vector<EpiX32<false>> ex32;
    std::vector<EpiY32<false>> ey32;
    std::vector<EpiX<true>> exc;
    std::vector<EpiY<true>> eyc;
    std::vector<EpiX32<true>> exc32;
    std::vector<EpiY32<true>> eyc32;
    std::vector<EpiDual> ed;
    std::vector<EpiPrimal> ep;
    std::vector<RedTask> red;
    for (size_t i = 0; i < b->ctxs.size(); ++i) {
        hpr_ctx *c = b->ctxs[i];
        sT64.push_back(sell_of(c->ST, false));
        sA64.push_back(sell_of(c->SA, false));
        sT32.push_back(sell_of(c->ST, true));
        sA32.push_back(sell_of(c->SA, true));
        ex.push_back(epi_x<false>(c, 0));
        ey.push_back(epi_y<false>(c, 0));
        ex32.push_back(epi_x32<false>(c, 0));
        ey32.push_back(epi_y32<false>(c, 0));
        exc.push_back(epi_x<true>(c, 0));
        eyc.push_back(epi_y<true>(c, 0));
        exc32.push_back(epi_x32<true>(c, 0));
        eyc32.push_back(epi_y32<true>(c, 0));
        ed.push_back(epi_dual(c));
        ep.push_back(epi_primal(c));
        const int nX = c->ST.rows ? c->ST.grid : 0, nY = c->SA.rows ? c->SA.grid : 0;
        const std::pair<int, int> qs[10] = {{Q_DX2, nX}, {Q_XX0, nX}, {Q_CX, nX}, {Q_BND, nX}, {Q_DY2, nY},
                                            {Q_YY0, nY}, {Q_BY, nY}, {Q_RD, nX}, {Q_RP, nY}, {Q_CROSS, nY}};
        for (const auto &q : qs)
            red.push_back(RedTask{c->partials, c->pstride, q.first, q.second, 0, c->ctl,
                                  b->scal_all + i * 2 * NQ});
    }
    auto put = [&](auto &h, auto **d) -> int {
        using T = typename std::remove_reference<decltype(h)>::type::value_type;
        if (alloc && cudaMalloc((void **)d, sizeof(T) * h.size()) != cudaSuccess) return HPR_ERR_NOMEM;
        if (cudaMemcpy(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess) return HPR_ERR_CUDA;
        return HPR_OK;
    };
    int st;
    if ((st = put(sT64, &b->sellT64)) || (st = put(sA64, &b->sellA64)) || (st = put(sT32, &b->sellT32)) ||
        (st = put(sA32, &b->sellA32)) || (st = put(ex, &b->ex)) || (st = put(ey, &b->ey)) ||
        (st = put(ex32, &b->ex32)) || (st = put(ey32, &b->ey32)) || (st = put(exc, &b->exc)) ||
        (st = put(eyc, &b->eyc)) || (st = put(exc32, &b->exc32)) || (st = put(eyc32, &b->eyc32)) ||
        (st = put(ed, &b->edual)) || (st = put(ep, &b->eprim)) || (st = put(red, &b->red)))
        return st;
    b->nred = (int)red.size();
    return HPR_OK;
}

template <class E, int MODE, int FORM>
int launch_multi(hpr_batch *b, const MultiTask *tasks, int ntasks, const SellArgs *sells, const E *epis, int it)
{
    if (ntasks == 0) return HPR_OK;
    k_sell_multi<E, MODE, FORM><<<ntasks, SELL_TB, 0, b->stream>>>(tasks, sells, epis, it);
    if (cudaGetLastError() != cudaSuccess) return HPR_ERR_CUDA;
    b->fused_launches += 1;
    return HPR_OK;
}

// every context's period of L iterations as fused launches: iterations 0 and L-1 in check
// mode (with the residual passes and reductions) for the contexts that check there, the
// others as normal iterations (each context's control block says which it takes part in)
int enqueue_fused(hpr_batch *b, int L, int forms)
{
    int st;
    const int nT = b->ntasksT, nA = b->ntasksA;
    for (int it = 0; it < L; ++it) {
        const bool chk = (it == 0 || it == L - 1), nrm = it < L - 1;
        if (chk && (forms & 1) && (st = launch_multi<EpiX<true>, 1, 0>(b, b->tasksT, nT, b->sellT64, b->exc, it))) return st;
        if (chk && (forms & 2) && (st = launch_multi<EpiX32<true>, 1, 1>(b, b->tasksT, nT, b->sellT32, b->exc32, it))) return st;
        if (nrm && (forms & 1) && (st = launch_multi<EpiX<false>, 0, 0>(b, b->tasksT, nT, b->sellT64, b->ex, it))) return st;
        if (nrm && (forms & 2) && (st = launch_multi<EpiX32<false>, 0, 1>(b, b->tasksT, nT, b->sellT32, b->ex32, it))) return st;
        if (chk && (forms & 1) && (st = launch_multi<EpiY<true>, 1, 0>(b, b->tasksA, nA, b->sellA64, b->eyc, it))) return st;
        if (chk && (forms & 2) && (st = launch_multi<EpiY32<true>, 1, 1>(b, b->tasksA, nA, b->sellA32, b->eyc32, it))) return st;
        if (nrm && (forms & 1) && (st = launch_multi<EpiY<false>, 0, 0>(b, b->tasksA, nA, b->sellA64, b->ey, it))) return st;
        if (nrm && (forms & 2) && (st = launch_multi<EpiY32<false>, 0, 1>(b, b->tasksA, nA, b->sellA32, b->ey32, it))) return st;
        if (chk) {
            if ((st = launch_multi<EpiDual, 1, -1>(b, b->tasksT, nT, b->sellT64, b->edual, it))) return st;
            if ((st = launch_multi<EpiPrimal, 1, -1>(b, b->tasksA, nA, b->sellA64, b->eprim, it))) return st;
            k_reduce_multi<<<b->nred, TB, 0, b->stream>>>(b->red, it);
            if (cudaGetLastError() != cudaSuccess) return HPR_ERR_CUDA;
            b->fused_launches += 1;
        }
    }
    return HPR_OK;
}

}  // namespace

extern "C" {

int hpr_batch_create(hpr_batch **out, int64_t count, hpr_ctx *const *ctxs, void *cuda_stream)
{
    if (!out) return HPR_ERR_ARG;
    *out = nullptr;
    if (count < 1 || count > (1 << 20) || !ctxs) {
        g_static_err = "hpr_batch_create: count outside [1, 2^20] or NULL context array";
        return HPR_ERR_ARG;
    }
    std::vector<hpr_ctx *> cs(ctxs, ctxs + count);
    for (size_t i = 0; i < cs.size(); ++i) {
        if (!cs[i] || cs[i]->batched || cs[i]->device != cs[0]->device) {
            g_static_err = "hpr_batch_create: NULL context, context already in a batch, or contexts on different devices";
            return HPR_ERR_ARG;
        }
        for (size_t j = 0; j < i; ++j)
            if (cs[j] == cs[i]) {
                g_static_err = "hpr_batch_create: a context appears twice";
                return HPR_ERR_ARG;
            }
    }
    hpr_batch *b = new (std::nothrow) hpr_batch();
    if (!b) return HPR_ERR_NOMEM;
    b->device = cs[0]->device;
    cudaSetDevice(b->device);
    auto fail = [&](int code, const char *what) {
        g_static_err = what;
        batch_free(b);
        delete b;
        return code;
    };
    if (cuda_stream) {
        b->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess)
            return fail(HPR_ERR_CUDA, "hpr_batch_create: cudaStreamCreate failed");
        b->own_stream = true;
    }
    for (hpr_ctx *c : cs) cudaStreamSynchronize(c->stream);
    b->ctxs = cs;
    // a fused phase that moves at least SMALL_PHASE_BYTES in total is bandwidth-bound: the
    // contexts' short-slice layouts (the small-phase rule) give way to the default layout
    {
        double sx = 0.0, sy = 0.0;
        for (hpr_ctx *c : cs) {
            sx += phase_bytes_x(c);
            sy += phase_bytes_y(c);
        }
        if (!batch_all_small(b))     // (a batch of single-CTA solves keeps the short slices)
            for (hpr_ctx *c : cs)
                if (relayout_for_throughput(c, sy >= SMALL_PHASE_BYTES, sx >= SMALL_PHASE_BYTES) != HPR_OK)
                    return fail(HPR_ERR_CUDA, "hpr_batch_create: relayout for throughput failed");
    }
    std::vector<MultiTask> tT = fused_tasks(cs, true), tA = fused_tasks(cs, false);
    int st = HPR_OK;
    if (cudaMalloc((void **)&b->scal_all, sizeof(double) * 2 * NQ * cs.size()) != cudaSuccess ||
        cudaMallocHost((void **)&b->scal_all_h, sizeof(double) * 2 * NQ * cs.size()) != cudaSuccess)
        return fail(HPR_ERR_NOMEM, "hpr_batch_create: check scalars could not be allocated");
    if ((st = upload_table(tT, &b->tasksT)) || (st = upload_table(tA, &b->tasksA)) ||
        (st = batch_tables(b, true)))
        return fail(st, "hpr_batch_create: device tables could not be allocated or copied");
    b->ntasksT = (int)tT.size();
    b->ntasksA = (int)tA.size();
    for (hpr_ctx *c : cs) {
        c->stream = b->stream;
        c->batched = true;
    }
    *out = b;
    return HPR_OK;
}

int hpr_batch_solve(hpr_batch *b, double tol)
{
    if (!b) return HPR_ERR_ARG;
    if (!(tol > 0.0)) {
        g_static_err = "hpr_batch_solve: tol must be > 0";
        return HPR_ERR_ARG;
    }
    cudaSetDevice(b->device);
    std::vector<hpr_ctx *> &cs = b->ctxs;
    for (hpr_ctx *c : cs) {
        if (c->opt.trace_iters > 0 || c->opt.check_every != cs[0]->opt.check_every) {
            g_static_err = "hpr_batch_solve: tracing is not available in a batch, and all contexts need the same check_every";
            return HPR_ERR_ARG;
        }
    }
    if (batch_all_small(b)) return batch_small(b, tol);
    const double t0 = now_s();
    b->periods = 0;
    b->fused_launches = 0;
    // power methods: each context on a stream of its worker thread, workers in parallel
    {
        const int W = (int)std::max<int64_t>(1, std::min<int64_t>(b->power_threads, (int64_t)cs.size()));
        std::vector<int> rc((size_t)W, HPR_OK);
        std::vector<std::thread> pool;
        for (int w = 0; w < W; ++w) {
            pool.emplace_back([&, w]() {
                cudaSetDevice(b->device);
                cudaStream_t ws = nullptr;
                if (cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) != cudaSuccess) {
                    rc[(size_t)w] = HPR_ERR_CUDA;
                    return;
                }
                for (size_t i = (size_t)w; i < cs.size() && rc[(size_t)w] == HPR_OK; i += (size_t)W) {
                    hpr_ctx *c = cs[i];
                    c->stream = ws;
                    rc[(size_t)w] = solve_begin(c, tol);
                    cudaStreamSynchronize(ws);
                    c->stream = b->stream;
                }
                cudaStreamDestroy(ws);
            });
        }
        for (auto &th : pool) th.join();
        for (int v : rc)
            if (v != HPR_OK) return v;
    }
    // every control block in one array for the solve (the contexts' own come back after it)
    size_t need = 0;
    for (hpr_ctx *c : cs) need = std::max(need, c->ctl_bytes);
    const size_t stride = (need + 255) & ~(size_t)255;
    if (stride > b->ctl_stride) {
        if (b->ctl_all) cudaFree(b->ctl_all);
        if (b->ctl_all_h) cudaFreeHost(b->ctl_all_h);
        b->ctl_all = b->ctl_all_h = nullptr;
        b->ctl_stride = 0;
        if (cudaMalloc((void **)&b->ctl_all, stride * cs.size()) != cudaSuccess ||
            cudaMallocHost((void **)&b->ctl_all_h, stride * cs.size()) != cudaSuccess) {
            g_static_err = "hpr_batch_solve: control blocks could not be allocated";
            return HPR_ERR_NOMEM;
        }
        b->ctl_stride = stride;
    }
    struct Saved { DevCtl *ctl, *ctl_h; size_t bytes; };
    std::vector<Saved> saved;
    for (size_t i = 0; i < cs.size(); ++i) {
        hpr_ctx *c = cs[i];
        saved.push_back({c->ctl, c->ctl_h, c->ctl_bytes});
        memset(b->ctl_all_h + i * b->ctl_stride, 0, b->ctl_stride);
        c->ctl = reinterpret_cast<DevCtl *>(b->ctl_all + i * b->ctl_stride);
        c->ctl_h = reinterpret_cast<DevCtl *>(b->ctl_all_h + i * b->ctl_stride);
    }
    auto restore = [&]() {
        for (size_t i = 0; i < cs.size(); ++i) {
            cs[i]->ctl = saved[i].ctl;
            cs[i]->ctl_h = saved[i].ctl_h;
            cs[i]->ctl_bytes = saved[i].bytes;
        }
    };
    int st = batch_tables(b, false);
    if (st) {
        restore();
        g_static_err = "hpr_batch_solve: device tables could not be refreshed";
        return st;
    }
    for (hpr_ctx *c : cs) c->ss.ctl_off = false;
    auto fail = [&](int code, const char *what) {
        cudaStreamSynchronize(b->stream);
        restore();
        if (what) g_static_err = what;
        return code;
    };
    for (;;) {
        std::vector<size_t> act;
        for (size_t i = 0; i < cs.size(); ++i)
            if (!cs[i]->ss.done) act.push_back(i);
        if (act.empty()) break;
        int forms = 0;
        for (hpr_ctx *c : cs) {
            if (c->ss.done) {                // once: its control block takes it out of fused launches
                if (!c->ss.ctl_off && (st = period_prepare(c, false))) return fail(st, nullptr);
                c->ss.ctl_off = true;
                continue;
            }
            if ((st = period_prepare(c, false))) return fail(st, nullptr);
            forms |= c->form == 1 ? 2 : 1;
        }
        const int L = cs[act[0]]->ss.L;
        for (size_t i : act)
            if (cs[i]->ss.L != L) return fail(HPR_ERR_STATE, "hpr_batch_solve: contexts out of step");
        if (cudaMemcpyAsync(b->ctl_all, b->ctl_all_h, b->ctl_stride * cs.size(), cudaMemcpyHostToDevice,
                            b->stream) != cudaSuccess)
            return fail(HPR_ERR_CUDA, "hpr_batch_solve: control block copy failed");
        const auto key = std::make_pair(L, forms);
        auto itg = b->graphs.find(key);
        if (itg == b->graphs.end()) {
            if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
                return fail(HPR_ERR_CUDA, "hpr_batch_solve: graph capture failed");
            const int64_t before = b->fused_launches;
            int rr = enqueue_fused(b, L, forms);
            b->graph_nodes[key] = b->fused_launches - before;
            b->fused_launches = before;
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(b->stream, &g);
            if (rr || e != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return fail(rr ? rr : HPR_ERR_CUDA, "hpr_batch_solve: graph capture failed");
            }
            cudaGraphExec_t ex = nullptr;
            e = cudaGraphInstantiate(&ex, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return fail(HPR_ERR_CUDA, "hpr_batch_solve: graph instantiation failed");
            itg = b->graphs.emplace(key, ex).first;
        }
        if (cudaGraphLaunch(itg->second, b->stream) != cudaSuccess)
            return fail(HPR_ERR_CUDA, "hpr_batch_solve: graph launch failed");
        b->fused_launches += b->graph_nodes[key];
        if (cudaMemcpyAsync(b->scal_all_h, b->scal_all, sizeof(double) * 2 * NQ * cs.size(),
                            cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
            cudaStreamSynchronize(b->stream) != cudaSuccess)
            return fail(HPR_ERR_CUDA, "hpr_batch_solve: CUDA error during a period");
        for (size_t i : act) {
            hpr_ctx *c = cs[i];
            memcpy(c->scal_h, b->scal_all_h + i * 2 * NQ, sizeof(double) * 2 * NQ);
            if ((st = period_after(c, now_s() - c->ss.t0))) return fail(st, nullptr);
        }
        b->periods++;
    }
    int worst = HPR_OK;
    for (hpr_ctx *c : cs) {
        st = solve_finish(c);
        if (st < 0) return fail(st, nullptr);
        if (st != HPR_OK) worst = st;
    }
    restore();
    b->solve_time = now_s() - t0;
    return worst;
}

int hpr_batch_stats(const hpr_batch *b, double *solve_time_s, int64_t *periods, int64_t *fused_launches)
{
    if (!b) return HPR_ERR_ARG;
    if (solve_time_s) *solve_time_s = b->solve_time;
    if (periods) *periods = b->periods;
    if (fused_launches) *fused_launches = b->fused_launches;
    return HPR_OK;
}

void hpr_batch_destroy(hpr_batch *b)
{
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_free(b);
    delete b;
}

}  // extern "C"


// ====================================================================== sigma policy network
namespace {

struct MlpBuffers {
    float *w = nullptr, *m = nullptr, *v = nullptr, *g = nullptr, *gpart = nullptr, *X = nullptr, *y = nullptr;
    __nv_bfloat16 *wb = nullptr;
    double *lpart = nullptr, *loss = nullptr;
    int *act = nullptr, *idx = nullptr;
    int max_ctas = 0;
    ~MlpBuffers()
    {
        void *p[] = {w, m, v, g, gpart, X, y, wb, lpart, loss, act, idx};
        for (void *q : p)
            if (q) cudaFree(q);
    }
};

int mlp_check_data(int64_t n, const float *X, const int32_t *act, const float *y)
{
    if (n < 1 || n > ((int64_t)1 << 26) || !X || (act && !y) || (!act && y)) return HPR_ERR_ARG;
    for (int64_t i = 0; i < n * hprmlp::IN; ++i)
        if (!std::isfinite(X[i])) return HPR_ERR_ARG;
    if (act)
        for (int64_t i = 0; i < n; ++i)
            if (act[i] < 0 || act[i] >= hprmlp::OUT || !std::isfinite(y[i])) return HPR_ERR_ARG;
    return HPR_OK;
}

// upload weights (and data) and make the BF16 copy
int mlp_setup(MlpBuffers &B, const float *w, int64_t n, const float *X, const int32_t *act, const float *y,
              int64_t batch)
{
    using namespace hprmlp;
    B.max_ctas = (int)std::min<int64_t>(592, std::max<int64_t>(1, (batch + 7) / 8));
    if (cudaMalloc((void **)&B.w, sizeof(float) * P) || cudaMalloc((void **)&B.m, sizeof(float) * P) ||
        cudaMalloc((void **)&B.v, sizeof(float) * P) || cudaMalloc((void **)&B.g, sizeof(float) * P) ||
        cudaMalloc((void **)&B.wb, sizeof(__nv_bfloat16) * P) ||
        cudaMalloc((void **)&B.gpart, sizeof(float) * (size_t)P * B.max_ctas) ||
        cudaMalloc((void **)&B.lpart, sizeof(double) * B.max_ctas) || cudaMalloc((void **)&B.loss, sizeof(double) * 2) ||
        cudaMalloc((void **)&B.X, sizeof(float) * (size_t)n * IN) || cudaMalloc((void **)&B.idx, sizeof(int) * (size_t)n))
        return HPR_ERR_NOMEM;
    if (act && (cudaMalloc((void **)&B.act, sizeof(int) * (size_t)n) || cudaMalloc((void **)&B.y, sizeof(float) * (size_t)n)))
        return HPR_ERR_NOMEM;
    if (cudaMemcpy(B.w, w, sizeof(float) * P, cudaMemcpyHostToDevice) ||
        cudaMemcpy(B.X, X, sizeof(float) * (size_t)n * IN, cudaMemcpyHostToDevice) ||
        cudaMemset(B.m, 0, sizeof(float) * P) || cudaMemset(B.v, 0, sizeof(float) * P))
        return HPR_ERR_CUDA;
    if (act && (cudaMemcpy(B.act, act, sizeof(int) * (size_t)n, cudaMemcpyHostToDevice) ||
                cudaMemcpy(B.y, y, sizeof(float) * (size_t)n, cudaMemcpyHostToDevice)))
        return HPR_ERR_CUDA;
    if (cudaFuncSetAttribute(k_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GRAD_SMEM)) return HPR_ERR_CUDA;
    k_to_bf16<<<26, 512>>>(B.w, B.wb);
    return cudaGetLastError() == cudaSuccess ? HPR_OK : HPR_ERR_CUDA;
}

// mean loss and gradient over samples idx[0 .. count) (idx NULL: the first count)
int mlp_grad_pass(MlpBuffers &B, const int *idx, int64_t count, double *loss_dst)
{
    using namespace hprmlp;
    const int ctas = (int)std::min<int64_t>(B.max_ctas, count);
    const int chunk = (int)((count + ctas - 1) / ctas);
    const int used = (int)((count + chunk - 1) / chunk);
    k_grad<<<used, TPB, GRAD_SMEM>>>(B.wb, B.X, B.act, B.y, idx, (int)count, chunk, B.gpart, B.lpart);
    k_reduce_grad<<<26, 512>>>(B.gpart, B.lpart, used, 1.0 / (double)count, B.g, loss_dst);
    return cudaGetLastError() == cudaSuccess ? HPR_OK : HPR_ERR_CUDA;
}

}  // namespace

extern "C" {

int hpr_mlp_param_count(void) { return hprmlp::P; }

int hpr_set_policy(hpr_ctx *ctx, const float *w)
{
    if (!ctx) return HPR_ERR_ARG;
    cudaSetDevice(ctx->device);
    if (!w) {
        if (ctx->policy_wb) cudaFree(ctx->policy_wb);
        ctx->policy_wb = nullptr;
        return HPR_OK;
    }
    for (int p = 0; p < hprmlp::P; ++p)
        if (!std::isfinite(w[p])) return fail_arg(ctx, HPR_ERR_ARG, "hpr_set_policy: non-finite weight");
    if (!ctx->policy_wb) DALLOC(ctx->policy_wb, hprmlp::P);
    if (!ctx->policy_w32) DALLOC(ctx->policy_w32, hprmlp::P);
    if (!ctx->policy_x) DALLOC(ctx->policy_x, hprmlp::IN);
    if (!ctx->policy_q) DALLOC(ctx->policy_q, hprmlp::OUT);
    CK(cudaMemcpyAsync(ctx->policy_w32, w, sizeof(float) * hprmlp::P, cudaMemcpyHostToDevice, ctx->stream));
    hprmlp::k_to_bf16<<<26, 512, 0, ctx->stream>>>(ctx->policy_w32, ctx->policy_wb);
    CKL();
    CK(cudaStreamSynchronize(ctx->stream));
    return HPR_OK;
}

int hpr_policy_features(const hpr_ctx *ctx, int64_t rec, float *out)
{
    if (!ctx || !out) return HPR_ERR_ARG;
    if (rec < 0 || rec >= (int64_t)ctx->checks.size())
        return fail_arg(const_cast<hpr_ctx *>(ctx), HPR_ERR_ARG, "hpr_policy_features: no such check record");
    policy_features(ctx->checks, rec, out);
    return HPR_OK;
}

int hpr_mlp_infer(const float *w, int64_t n, const float *X, float *Q)
{
    if (!w || !Q || mlp_check_data(n, X, nullptr, nullptr)) {
        g_static_err = "hpr_mlp_infer: NULL array, n outside [1, 2^26] or non-finite input";
        return HPR_ERR_ARG;
    }
    MlpBuffers B;
    int st = mlp_setup(B, w, n, X, nullptr, nullptr, 1);
    if (st) { g_static_err = "hpr_mlp_infer: device setup failed"; return st; }
    float *dQ = nullptr;
    if (cudaMalloc((void **)&dQ, sizeof(float) * (size_t)n * hprmlp::OUT)) return HPR_ERR_NOMEM;
    hprmlp::k_infer<<<(int)std::min<int64_t>(n, 4096), hprmlp::TPB>>>(B.wb, B.X, (int)n, dQ);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(Q, dQ, sizeof(float) * (size_t)n * hprmlp::OUT, cudaMemcpyDeviceToHost);
    cudaFree(dQ);
    if (e != cudaSuccess) { g_static_err = "hpr_mlp_infer: CUDA error"; return HPR_ERR_CUDA; }
    return HPR_OK;
}

int hpr_mlp_grad(const float *w, int64_t n, const float *X, const int32_t *act, const float *y, float *grad,
                 double *loss)
{
    if (!w || !grad || !act || mlp_check_data(n, X, act, y)) {
        g_static_err = "hpr_mlp_grad: NULL array, n outside [1, 2^26], action outside [0, 5) or non-finite input";
        return HPR_ERR_ARG;
    }
    MlpBuffers B;
    int st = mlp_setup(B, w, n, X, act, y, n);
    if (st) { g_static_err = "hpr_mlp_grad: device setup failed"; return st; }
    if ((st = mlp_grad_pass(B, nullptr, n, B.loss))) return st;
    if (cudaMemcpy(grad, B.g, sizeof(float) * hprmlp::P, cudaMemcpyDeviceToHost) != cudaSuccess) return HPR_ERR_CUDA;
    if (loss && cudaMemcpy(loss, B.loss, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) return HPR_ERR_CUDA;
    return HPR_OK;
}

int hpr_mlp_train(float *w, int64_t n, const float *X, const int32_t *act, const float *y, int64_t epochs,
                  int64_t batch, double lr, uint64_t seed, double *epoch_loss)
{
    if (!w || !act || mlp_check_data(n, X, act, y) || epochs < 0 || epochs > 100000 || batch < 1 ||
        !(lr > 0.0) || !(lr < 1.0)) {
        g_static_err = "hpr_mlp_train: bad arguments (NULL array, n outside [1, 2^26], action outside [0, 5), "
                       "non-finite input, epochs outside [0, 1e5], batch < 1 or lr outside (0, 1))";
        return HPR_ERR_ARG;
    }
    batch = std::min(batch, n);
    MlpBuffers B;
    int st = mlp_setup(B, w, n, X, act, y, batch);
    if (st) { g_static_err = "hpr_mlp_train: device setup failed"; return st; }
    const int64_t steps_per_epoch = (n + batch - 1) / batch;
    double *hist = nullptr;
    if (cudaMalloc((void **)&hist, sizeof(double) * (size_t)std::max<int64_t>(1, epochs * steps_per_epoch)))
        return HPR_ERR_NOMEM;
    std::vector<int> perm((size_t)n);
    uint64_t rng = seed;
    int64_t t = 0;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int64_t ep = 0; ep < epochs && st == HPR_OK; ++ep) {
        // Fisher-Yates with SplitMix64 draws: a fixed sample order per (seed, epoch)
        for (int64_t i = 0; i < n; ++i) perm[(size_t)i] = (int)i;
        for (int64_t i = n - 1; i > 0; --i) {
            const int64_t r = (int64_t)(splitmix64_next(rng) % (uint64_t)(i + 1));
            std::swap(perm[(size_t)i], perm[(size_t)r]);
        }
        if (cudaMemcpy(B.idx, perm.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice) != cudaSuccess) {
            st = HPR_ERR_CUDA;
            break;
        }
        for (int64_t s0 = 0; s0 < n && st == HPR_OK; s0 += batch) {
            const int64_t cnt = std::min(batch, n - s0);
            st = mlp_grad_pass(B, B.idx + s0, cnt, hist + t);
            ++t;
            const float c1 = 1.f - std::pow(b1, (float)t), c2 = 1.f - std::pow(b2, (float)t);
            hprmlp::k_adam<<<26, 512>>>(B.w, B.m, B.v, B.g, (float)lr, b1, b2, eps, c1, c2, B.wb);
            if (st == HPR_OK && cudaGetLastError() != cudaSuccess) st = HPR_ERR_CUDA;
        }
    }
    if (st == HPR_OK && cudaMemcpy(w, B.w, sizeof(float) * hprmlp::P, cudaMemcpyDeviceToHost) != cudaSuccess)
        st = HPR_ERR_CUDA;
    if (st == HPR_OK && epoch_loss && epochs > 0) {
        std::vector<double> h((size_t)(epochs * steps_per_epoch));
        if (cudaMemcpy(h.data(), hist, sizeof(double) * h.size(), cudaMemcpyDeviceToHost) != cudaSuccess) {
            st = HPR_ERR_CUDA;
        } else {
            for (int64_t ep = 0; ep < epochs; ++ep) {
                double sum = 0.0;
                for (int64_t k = 0; k < steps_per_epoch; ++k) sum += h[(size_t)(ep * steps_per_epoch + k)];
                epoch_loss[ep] = sum / (double)steps_per_epoch;
            }
        }
    }
    cudaFree(hist);
    if (st) g_static_err = "hpr_mlp_train: CUDA error";
    return st;
}

}  // extern "C"

// ====================================================================== allocation-free power method
//
// For callers that must not allocate device memory (they run under a memory budget
// owned by someone else, inside a capture region, or on a pool whose allocator is not
// theirs).  The LP is theirs, already on the device; this entry point needs only the
// per-CTA partial sums, a few reduced scalars and the power-method control block, and
// keeps them in one fixed array in device global memory that is part of the library
// image.  Every device that loads the library holds that array until the process
// exits; every call on a device shares it.

namespace {

constexpr int NA_SLOTS = 1024;                           // CTAs per reduction, at most
constexpr int NA_PARTIALS = NQ * NA_SLOTS;               // per-CTA partial sums
constexpr int NA_SCAL = NA_PARTIALS;                     // NQ reduced scalars
constexpr int NA_CTL = NA_SCAL + NQ;                     // PowCtl (6 doubles)
constexpr int NA_INV = NA_CTL + 8;                       // 1 / ||u0||
constexpr int NA_DOUBLES = NA_INV + 8;                   // 16,432 doubles = 131,456 bytes

static __device__ __align__(256) double g_noalloc_scratch[NA_DOUBLES];

// Warp-per-row variant of k_spmv_norm: out = M xin, partial ||out||^2 per CTA.  No tile
// schedule is needed, so the caller's plain CSR arrays are enough.
__global__ void __launch_bounds__(TB) k_rows_spmv_norm(int rows, const int *__restrict__ rp,
                                                       const int *__restrict__ ci,
                                                       const double *__restrict__ val,
                                                       const double *__restrict__ xin, double *out,
                                                       double *partials, int pstride, int q,
                                                       const PowCtl *pc)
{
    __shared__ double red[TB / 32];
    if (pc->done) return;
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (TB / 32);
    double p = 0.0;
    for (int r = blockIdx.x * (TB / 32) + (threadIdx.x >> 5); r < rows; r += warps) {
        double s = 0.0;
        for (int k = rp[r] + lane; k < rp[r + 1]; k += 32) s = fma(val[k], __ldg(xin + ci[k]), s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            out[r] = s;
            p = fma(s, s, p);
        }
    }
    const double t = block_sum(p, red);
    if (threadIdx.x == 0) partials[q * pstride + blockIdx.x] = t;
}

// start vector u_i = 2 U_i - 1 (SplitMix64), grid-stride, partial ||u||^2 per CTA
__global__ void __launch_bounds__(TB) k_rows_pow_start(int m, uint64_t seed, double *u,
                                                       double *partials, int pstride)
{
    __shared__ double red[TB / 32];
    double p = 0.0;
    for (int i = blockIdx.x * TB + threadIdx.x; i < m; i += gridDim.x * TB) {
        const double v = 2.0 * ((double)(splitmix64_at(seed, (uint64_t)i) >> 11) * 0x1.0p-53) - 1.0;
        u[i] = v;
        p = fma(v, v, p);
    }
    const double s = block_sum(p, red);
    if (threadIdx.x == 0) partials[Q_V2 * pstride + blockIdx.x] = s;
}

std::mutex g_na_mutex;
double *g_na_ptr[64] = {nullptr};   // device address of g_noalloc_scratch, per device
thread_local std::string g_na_err;

int na_fail(int code, const std::string &msg)
{
    g_na_err = msg;
    g_static_err = g_na_err.c_str();
    return code;
}

int na_fail_cuda(cudaError_t e, const char *what)
{
    (void)cudaGetLastError();
    return na_fail(HPR_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace

extern "C" int hpr_power_noalloc(int64_t m, int64_t n, const int32_t *A_row_ptr,
                                 const int32_t *A_col_idx, const double *A_val,
                                 const int32_t *At_row_ptr, const int32_t *At_col_idx,
                                 const double *At_val, uint64_t seed, int64_t max_iter,
                                 double tol, double *u, double *s, void *cuda_stream,
                                 double *lambda, int64_t *iters)
{
    if (m < 1 || n < 1 || m > (int64_t)INT32_MAX - 1 || n > (int64_t)INT32_MAX - 1)
        return na_fail(HPR_ERR_ARG, "hpr_power_noalloc: m and n must be in [1, 2^31 - 2]");
    if (!A_row_ptr || !A_col_idx || !A_val || !At_row_ptr || !At_col_idx || !At_val || !u || !s)
        return na_fail(HPR_ERR_ARG, "hpr_power_noalloc: NULL device pointer");
    if (max_iter < 1 || max_iter > (int64_t)INT32_MAX || !(tol >= 0.0))
        return na_fail(HPR_ERR_ARG, "hpr_power_noalloc: need 1 <= max_iter < 2^31 and tol >= 0");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail_cuda(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return na_fail(HPR_ERR_NO_DEVICE, "hpr_power_noalloc: device index above 63");
    double *base = nullptr;
    {
        // one-time set-up per device, with that device current: the device address of the
        // scratch array (its host-side name is not a device address)
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (!g_na_ptr[dev]) {
            e = cudaGetSymbolAddress((void **)&g_na_ptr[dev], g_noalloc_scratch);
            if (e != cudaSuccess) {
                g_na_ptr[dev] = nullptr;
                return na_fail_cuda(e, "cudaGetSymbolAddress(scratch)");
            }
        }
        base = g_na_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    double *partials = base, *scal = base + NA_SCAL, *inv = base + NA_INV;
    PowCtl *pc = reinterpret_cast<PowCtl *>(base + NA_CTL);
    const int gm = (int)std::min<int64_t>(NA_SLOTS, std::max<int64_t>(1, (m + TB - 1) / TB));
    const int gA = (int)std::min<int64_t>(NA_SLOTS, std::max<int64_t>(1, (m + 7) / 8));
    const int gT = (int)std::min<int64_t>(NA_SLOTS, std::max<int64_t>(1, (n + 7) / 8));

    // control block: every field that a call reads is written first (the array keeps
    // the previous call's contents)
    PowCtl h{};
    h.tol = tol;
    h.max_iter = (int)max_iter;
    e = cudaMemcpyAsync(pc, &h, sizeof h, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return na_fail_cuda(e, "cudaMemcpyAsync(control)");

    RedSpec r1{};
    r1.nq = 1;
    r1.q[0] = Q_V2;
    r1.cnt[0] = gm;
    k_rows_pow_start<<<gm, TB, 0, st>>>((int)m, seed, u, partials, NA_SLOTS);
    k_reduce<<<1, TB, 0, st>>>(partials, NA_SLOTS, r1, scal, nullptr);
    k_inv_sqrt_scalar<<<1, 1, 0, st>>>(scal, Q_V2, inv);
    k_scale_vec<<<gm, TB, 0, st>>>((int)m, u, u, nullptr, inv);
    e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail_cuda(e, "kernel launch");

    RedSpec rs{}, rw{};
    rs.nq = 1; rs.q[0] = Q_S2; rs.cnt[0] = gT;
    rw.nq = 1; rw.q[0] = Q_W2; rw.cnt[0] = gA;
    const int BATCH = 16;
    for (int64_t done_steps = 0; done_steps <= max_iter; done_steps += BATCH) {
        for (int k = 0; k < BATCH; ++k) {
            // s = A^T u, lambda_k = ||s||^2, then w = A s written over u and normalised
            k_rows_spmv_norm<<<gT, TB, 0, st>>>((int)n, At_row_ptr, At_col_idx, At_val, u, s,
                                                partials, NA_SLOTS, Q_S2, pc);
            k_reduce<<<1, TB, 0, st>>>(partials, NA_SLOTS, rs, scal, &pc->done);
            k_pow_after_s<<<1, 1, 0, st>>>(pc, scal);
            k_rows_spmv_norm<<<gA, TB, 0, st>>>((int)m, A_row_ptr, A_col_idx, A_val, s, u,
                                                partials, NA_SLOTS, Q_W2, pc);
            k_reduce<<<1, TB, 0, st>>>(partials, NA_SLOTS, rw, scal, &pc->done);
            k_pow_after_w<<<1, 1, 0, st>>>(pc, scal);
            k_scale_vec<<<gm, TB, 0, st>>>((int)m, u, u, pc, nullptr);
            k_pow_finish<<<1, 1, 0, st>>>(pc);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return na_fail_cuda(e, "kernel launch");
        e = cudaMemcpyAsync(&h, pc, sizeof h, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return na_fail_cuda(e, "reading the control block");
        if (h.done) break;
    }
    if (lambda) *lambda = h.lam;
    if (iters) *iters = h.k;
    if (!std::isfinite(h.lam) || !(h.lam > 0.0))
        return na_fail(HPR_ERR_NUMERIC, "hpr_power_noalloc: non-positive lambda");
    return HPR_OK;
}
