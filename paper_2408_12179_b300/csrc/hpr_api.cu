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
//
// One translation unit in five files: this one (context, layouts, launch helpers, power
// method, preprocessing, hpr_create and the option calls), then hpr_api_solve.cuh (the
// solve on both paths and the result calls), hpr_api_batch.cuh (batched solves),
// hpr_api_policy.cuh (the sigma policy network) and hpr_api_noalloc.cuh (the
// allocation-free power method), included at the end.
#include "hpr.h"
#include "hpr_device.cuh"
#include "hpr_mlp.cuh"
#include "hpr_small.cuh"
#include "hpr_grid.cuh"
#include "hpr_cluster.cuh"
#include "hpr_tiles.cuh"

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
    int cols = 0;                 // length of the vectors it gathers (columns of the matrix)
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

// A^T in the gather-tiled layout of the x phase (device arrays; see k_tile_part)
struct TileDev {
    int nblk = 0;                 // blocks of y (0: the layout is not built)
    int grid = 0;                 // CTAs of k_tile_part (one per SM)
    int glen_max = 0;             // entries of the longest block (its shared memory / 8)
    int64_t entries = 0, nsub = 0;   // stored entries (with padding); sub-rows = slots of P
    int *cta_blk = nullptr, *bstart = nullptr, *ustart = nullptr, *wstart = nullptr;
    int4 *smeta = nullptr;
    int *oslot = nullptr, *slot_ptr = nullptr, *src = nullptr;
    unsigned short *col = nullptr;
    double *val = nullptr, *P = nullptr;
    unsigned *ctr = nullptr;
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
    // the last restart (the checkpoint of hpr_get_state): its iteration count, sigma and
    // form; the anchors x0, y0 keep its w_bar for the whole inner loop
    int64_t k_restart = 0;
    double sigma_restart = 1.0;
    int form_restart = 0;
};

// header of a checkpoint blob (hpr_get_state / hpr_set_state), followed by the anchors
// x0 (n doubles) and y0 (m doubles) in the internal (scaled, renumbered) order
struct StateHdr {
    uint64_t magic;
    int64_t n, m, m1, nnz, precision, check_every;
    double beta_b, beta_c, norm_b, norm_c;   // the scaled LP's fingerprint
    int64_t k, r, form, power_iters;
    double sigma, lambda, power_rel_change;
};
constexpr uint64_t STATE_MAGIC = 0x4850525354415401ull;   // "HPRSTAT" and the layout version 1

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
    TileDev TX;                   // A^T in the gather-tiled layout (x phase), if built
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
    float *x032 = nullptr, *y032 = nullptr;   // FP32 copies of the anchors (FP32 form)
    float *cp32 = nullptr, *lp32 = nullptr, *up32 = nullptr, *bp32 = nullptr;   // and of the data
    float *cp32lo = nullptr, *bp32lo = nullptr;   // c, b as double-float pairs (hi above, lo here)
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
    unsigned *pow_ticket = nullptr;   // last-CTA tickets of the two power-method launches
    int64_t pow_ticket_len = 0;
    double *trace = nullptr;
    int64_t trace_n = 0;
    int64_t trace_written = 0;

    std::map<GraphKey, cudaGraphExec_t> graphs;
    std::map<GraphKey, int64_t> graph_launches;   // kernel nodes per captured period
    cudaGraphExec_t pow_graph = nullptr;
    int64_t pow_graph_launches = 0;   // kernels of one launch of pow_graph

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
    // host-side fault injection (environment, read at hpr_create; 0: off): the
    // fault_alloc-th device or pinned allocation of this context reports out-of-memory, and
    // the scalars of the fault_nan_check-th check period read back as NaN
    int64_t fault_alloc = 0, alloc_count = 0, fault_nan_check = 0, check_count = 0;

    // results
    bool solved = false;
    bool have_power = false;
    double lambda = 0.0;
    int64_t power_iters = 0;
    double power_time = 0.0;
    double power_rel_change = 0.0;   // the power method's last relative change of lambda
    hpr_info info{};
    SolveState ss;
    __nv_bfloat16 *policy_wb = nullptr;   // sigma policy network (BF16), its input and output
    float *policy_w32 = nullptr, *policy_x = nullptr, *policy_q = nullptr;
    hpr_check_record *small_recs = nullptr;   // persistent path: its check records and results
    double *small_out = nullptr;
    int small_cap = 0;
    hprsmall::SmallArgs *small_args = nullptr; // persistent path: device copy of its arguments
    double *grid_partials = nullptr;          // persistent grid path: CTA sums, barrier state
    hprgrid::GridBar *grid_bar = nullptr;
    int grid_ctas_used = 0;                   // CTAs of the last persistent grid or cluster solve
    int path_used = 0;                        // the path of the last solve (hpr_info.path)
    bool resume_pending = false;              // hpr_set_state: the next solve starts from it
    StateHdr resume_hdr{};
    std::vector<double> resume_x0, resume_y0;
    int64_t grid_ctas_env = 0;                // HPR_GRID_CTAS: CTA count of that path (0: by size)
    int64_t fault_barrier = 0;                // HPR_FAULT_BARRIER=n: a CTA skips barrier n-1
    bool batched = false;         // owned by a batch: solved only through hpr_batch_solve
    std::vector<hpr_check_record> checks;
    std::string err;
};

namespace {

// last error of a context-free call, per host thread (each thread reads only its own
// messages, which live in thread-local storage of the thread that wrote them)
thread_local const char *g_static_err = "no context";

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

// whether this allocation is the one HPR_FAULT_ALLOC asks to fail
bool fault_now(hpr_ctx *ctx)
{
    return ctx && ctx->fault_alloc > 0 && ++ctx->alloc_count == ctx->fault_alloc;
}

#define CKA(call)                                                                 \
    do {                                                                          \
        if (fault_now(ctx))                                                       \
            return fail_cuda(ctx, cudaErrorMemoryAllocation, #call " (HPR_FAULT_ALLOC)", __LINE__); \
        CK(call);                                                                 \
    } while (0)

template <class T>
int dalloc(hpr_ctx *ctx, T **p, int64_t count)
{
    size_t bytes = sizeof(T) * (size_t)(count > 0 ? count : 1);
    if (fault_now(ctx)) {
        *p = nullptr;
        return fail_cuda(ctx, cudaErrorMemoryAllocation, "cudaMalloc (HPR_FAULT_ALLOC)", __LINE__);
    }
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
    // pass 1: the slices (rows, lanes, steps) and where each one's entries start
    h.srow.push_back(0);
    h.sptr.push_back(0);
    size_t total = 0;
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
            total += (size_t)32 * steps;
            h.slg.push_back((unsigned char)lg);
            h.srow.push_back(r1);
            h.sptr.push_back((int)total);
            h.nslices++;
            scost.push_back((double)steps + 2.0 + lg + 8.0 * (r1 - r) / 32.0);
        }
    }
    gfirst.push_back(h.nslices);
    // pass 2: every slice's entries into its own range (padding: column 0, no source), on
    // up to 16 host threads over contiguous runs of slices of about equal size
    h.col.assign(total, 0);
    h.src.assign(total, -1);
    auto fill = [&](int s0, int s1) {
        for (int sl = s0; sl < s1; ++sl) {
            const int lg = h.slg[(size_t)sl], L = 1 << lg;
            const int r = h.srow[(size_t)sl], r1 = h.srow[(size_t)sl + 1];
            const size_t base = (size_t)h.sptr[(size_t)sl];
            for (int q = 0; q < r1 - r; ++q) {
                const int orow = perm[(size_t)(r + q)];
                for (int e = 0, p = rp[(size_t)orow]; p < rp[(size_t)orow + 1]; ++p, ++e) {
                    const size_t at = base + (size_t)(e / L) * 32 + (size_t)(q * L + e % L);
                    h.col[at] = icol[(size_t)ci[(size_t)p]];
                    h.src[at] = p;
                }
            }
        }
    };
    const int nthr = total < ((size_t)1 << 20)
                         ? 1
                         : (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    if (nthr == 1) {
        fill(0, h.nslices);
    } else {
        std::vector<std::thread> pool;
        int s0 = 0;
        for (int t = 0; t < nthr && s0 < h.nslices; ++t) {
            const size_t goal = total * (size_t)(t + 1) / (size_t)nthr;
            int s1 = s0;
            while (s1 < h.nslices && (t == nthr - 1 || (size_t)h.sptr[(size_t)s1] < goal)) ++s1;
            pool.emplace_back(fill, s0, s1);
            s0 = s1;
        }
        for (auto &th : pool) th.join();
    }
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

// Gather-tiled layout of a matrix whose phase gathers a vector of `cols` entries (see
// k_tile_part): the gathered vector is cut into blocks of at most `tile_len` consecutive
// entries (even, so every block starts 16-byte aligned), balanced by stored entries; each
// block gets CTAs of the grid in proportion to its entries (at least one); the entries of
// each block form a sub-matrix whose rows (sub-rows: the rows with an entry in the block,
// in renumbered order) take the sliced-ELL layout of build_sell with column offsets within
// the block.  Slot q of P holds a sub-row's sum; row r owns slots slot_ptr[r] ..
// slot_ptr[r+1]-1, in block order.  A work unit is a run of consecutive slices of one block.
// Rows are in the order perm, columns renamed by icol (the renumbering of the sliced-ELL
// layout).  Returns false (layout not built) when the blocks would outnumber the grid's CTAs
// or k_tile_epi's counter reset, or when the layout's offsets would not fit in 32 bits.
//
// Work units of the tiled layout: runs of slices of one block, each slice costing its steps
// + 4; a block's units are sized so that each warp of its CTAs gets about TILE_UNITS_PER_WARP
// of them (at least TILE_UNIT_MIN)
constexpr int TILE_UNITS_PER_WARP = 4;
constexpr int TILE_UNIT_MIN = 12;

struct TileHost {
    int nblk = 0;
    std::vector<int> bstart, ustart, cta_blk, wstart, srow, sptr, oslot, slot_ptr, src;
    std::vector<unsigned char> slg;
    std::vector<int4> smeta;         // per slice: srow, sptr, steps, slg | sub-rows << 8
    std::vector<unsigned short> col;
    int glen_max = 0;
};

bool build_tiles(const std::vector<int> &rp, const std::vector<int> &ci, int rows,
                 const std::vector<int> &perm, const std::vector<int> &icol, int cols,
                 int tile_len, int grid, int steps_max, double unit_cost, TileHost &h)
{
    tile_len &= ~1;
    if (rows < 1 || cols < 1 || tile_len < 2 || tile_len > 65536 || grid < 1) return false;
    const int64_t nnz = rp[(size_t)rows];
    std::vector<int64_t> cnt((size_t)cols, 0);
    for (int64_t p = 0; p < nnz; ++p) cnt[(size_t)icol[(size_t)ci[(size_t)p]]]++;
    // block boundaries: cut at an even column once the block holds its share of the
    // entries, or at tile_len columns
    const int goal = (int)std::min<int64_t>(grid, ((int64_t)cols + tile_len - 1) / tile_len);
    h.bstart.assign(1, 0);
    {
        int64_t acc = 0;
        int start = 0;
        for (int c = 0; c < cols; ++c) {
            if (c > start && (c & 1) == 0) {
                const int b = (int)h.bstart.size() - 1;
                const bool full = c - start >= tile_len;
                const bool share = b + 1 < goal && (double)acc >= (double)nnz * (b + 1) / goal;
                if (full || share) {
                    h.bstart.push_back(c);
                    start = c;
                }
            }
            acc += cnt[(size_t)c];
        }
        h.bstart.push_back(cols);
    }
    const int nblk = (int)h.bstart.size() - 1;
    if (nblk > grid || nblk > TILE_MAX_BLOCKS) return false;
    h.nblk = nblk;
    std::vector<int> colblk((size_t)cols);
    std::vector<int64_t> bnnz((size_t)nblk, 0);
    for (int b = 0; b < nblk; ++b) {
        h.glen_max = std::max(h.glen_max, h.bstart[(size_t)b + 1] - h.bstart[(size_t)b]);
        for (int c = h.bstart[(size_t)b]; c < h.bstart[(size_t)b + 1]; ++c) {
            colblk[(size_t)c] = b;
            bnnz[(size_t)b] += cnt[(size_t)c];
        }
    }
    // CTAs per block: one each, the rest one at a time to the block with the most entries
    // per CTA
    std::vector<int> ncta((size_t)nblk, 1);
    for (int g = nblk; g < grid; ++g) {
        int best = 0;
        for (int b = 1; b < nblk; ++b)
            if ((double)bnnz[(size_t)b] / ncta[(size_t)b] > (double)bnnz[(size_t)best] / ncta[(size_t)best]) best = b;
        ncta[(size_t)best]++;
    }
    h.cta_blk.clear();
    for (int b = 0; b < nblk; ++b) h.cta_blk.insert(h.cta_blk.end(), (size_t)ncta[(size_t)b], b);
    // the sub-matrices (CSR, rows in renumbered order) and the slots of each row
    std::vector<std::vector<int>> brow((size_t)nblk), brp((size_t)nblk), bci((size_t)nblk), bpos((size_t)nblk);
    for (int b = 0; b < nblk; ++b) {
        bci[(size_t)b].reserve((size_t)bnnz[(size_t)b]);
        bpos[(size_t)b].reserve((size_t)bnnz[(size_t)b]);
    }
    std::vector<int> last((size_t)nblk, -1);
    h.slot_ptr.assign((size_t)rows + 1, 0);
    for (int r = 0; r < rows; ++r) {
        const int orow = perm[(size_t)r];
        int nb = 0;
        for (int p = rp[(size_t)orow]; p < rp[(size_t)orow + 1]; ++p) {
            const int c = icol[(size_t)ci[(size_t)p]];
            const int b = colblk[(size_t)c];
            if (last[(size_t)b] != r) {
                last[(size_t)b] = r;
                brow[(size_t)b].push_back(r);
                brp[(size_t)b].push_back((int)bci[(size_t)b].size());
                ++nb;
            }
            bci[(size_t)b].push_back(c - h.bstart[(size_t)b]);
            bpos[(size_t)b].push_back(p);
        }
        h.slot_ptr[(size_t)r + 1] = h.slot_ptr[(size_t)r] + nb;
    }
    for (int b = 0; b < nblk; ++b) brp[(size_t)b].push_back((int)bci[(size_t)b].size());
    // slot of each sub-row: its row's slots are taken in block order
    std::vector<std::vector<int>> bslot((size_t)nblk);
    {
        std::vector<int> fill(h.slot_ptr.begin(), h.slot_ptr.end() - 1);
        for (int b = 0; b < nblk; ++b) {
            bslot[(size_t)b].resize(brow[(size_t)b].size());
            for (size_t q = 0; q < brow[(size_t)b].size(); ++q)
                bslot[(size_t)b][q] = fill[(size_t)brow[(size_t)b][q]]++;
        }
    }
    // sliced ELL of each sub-matrix (blocks in parallel on up to 16 host threads)
    std::vector<SellHost> bh((size_t)nblk);
    std::vector<std::vector<int>> bperm((size_t)nblk);
    auto lay = [&](int b) {
        const int nr = (int)brow[(size_t)b].size();
        const int len = h.bstart[(size_t)b + 1] - h.bstart[(size_t)b];
        std::vector<int> ident((size_t)len);
        for (int c = 0; c < len; ++c) ident[(size_t)c] = c;
        bperm[(size_t)b] = order_by_length(brp[(size_t)b], nr);
        bh[(size_t)b] = build_sell(brp[(size_t)b], bci[(size_t)b], nr, bperm[(size_t)b], ident, steps_max, unit_cost);
    };
    {
        const int nthr = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
        std::vector<std::thread> pool;
        for (int t = 0; t < std::min(nthr, nblk); ++t)
            pool.emplace_back([&, t] {
                for (int b = t; b < nblk; b += nthr) lay(b);
            });
        for (auto &th : pool) th.join();
    }
    // the concatenated offsets are 32-bit: a layout whose stored entries (padding included)
    // or sub-rows reach 2^31 - 1 is not built
    {
        int64_t ents = 0, subs = 0;
        for (int b = 0; b < nblk; ++b) {
            ents += (int64_t)bh[(size_t)b].col.size();
            subs += (int64_t)brow[(size_t)b].size();
        }
        if (ents >= (int64_t)INT32_MAX || subs >= (int64_t)INT32_MAX) return false;
    }
    // concatenation: slices, entries, sub-rows and units of block b follow those of b - 1
    h.ustart.assign(1, 0);
    h.wstart.clear();
    h.smeta.clear();
    h.srow.assign(1, 0);
    h.sptr.assign(1, 0);
    h.slg.clear();
    h.oslot.clear();
    h.col.clear();
    h.src.clear();
    int slice0 = 0, sub0 = 0, ent0 = 0;
    for (int b = 0; b < nblk; ++b) {
        const SellHost &H = bh[(size_t)b];
        int64_t total = 0;
        for (int sl = 0; sl < H.nslices; ++sl) total += ((H.sptr[(size_t)sl + 1] - H.sptr[(size_t)sl]) >> 5) + 4;
        const int64_t warps = (int64_t)ncta[(size_t)b] * (TILE_TB / 32) * TILE_UNITS_PER_WARP;
        const int64_t unit_target = std::max<int64_t>(TILE_UNIT_MIN, (total + warps - 1) / warps);
        int units = 0;
        int64_t cost = 0;
        for (int sl = 0; sl < H.nslices; ++sl) {
            if (cost == 0) {
                h.wstart.push_back(slice0 + sl);
                ++units;
            }
            const int steps = (H.sptr[(size_t)sl + 1] - H.sptr[(size_t)sl]) >> 5;
            cost += steps + 4;
            if (cost >= unit_target) cost = 0;
            h.smeta.push_back(make_int4(sub0 + H.srow[(size_t)sl], ent0 + H.sptr[(size_t)sl], steps,
                                        (int)H.slg[(size_t)sl] | ((H.srow[(size_t)sl + 1] - H.srow[(size_t)sl]) << 8)));
            h.srow.push_back(sub0 + H.srow[(size_t)sl + 1]);
            h.sptr.push_back(ent0 + H.sptr[(size_t)sl + 1]);
            h.slg.push_back(H.slg[(size_t)sl]);
        }
        h.ustart.push_back(h.ustart.back() + units);
        for (size_t t = 0; t < brow[(size_t)b].size(); ++t)
            h.oslot.push_back(bslot[(size_t)b][(size_t)bperm[(size_t)b][t]]);
        for (size_t e = 0; e < H.col.size(); ++e) {
            h.col.push_back((unsigned short)H.col[e]);
            h.src.push_back(H.src[e] < 0 ? -1 : bpos[(size_t)b][(size_t)H.src[e]]);
        }
        slice0 += H.nslices;
        sub0 += (int)brow[(size_t)b].size();
        ent0 += (int)H.col.size();
    }
    h.wstart.push_back(slice0);
    return true;
}

void free_tiles(TileDev &T)
{
    void *p[] = {T.cta_blk, T.bstart, T.ustart, T.wstart, T.smeta, T.oslot, T.slot_ptr, T.src,
                 T.col, T.val, T.P, T.ctr};
    for (void *q : p)
        if (q) cudaFree(q);
    T = TileDev{};
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
                   c->SA.val32, c->ST.val32, c->x32, c->xhat32, c->y32, c->x032, c->y032,
                   c->cp32, c->lp32, c->up32, c->bp32, c->cp32lo, c->bp32lo,
                   c->perm_r, c->perm_c, c->ineq, c->bp, c->cp, c->lp, c->up, c->wrp, c->wcp,
                   c->unperm, c->Dr, c->Dc, c->wr, c->wc, c->b_s, c->c_s,
                   c->l_s, c->u_s, c->l_o, c->u_o, c->x, c->x0, c->xhat, c->xbar,
                   c->zbar, c->dx, c->y, c->y0, c->ybar, c->dy, c->xo, c->yo, c->zo,
                   c->partials, c->scal, c->ctl, c->pctl, c->trace, c->policy_wb, c->policy_w32,
                   c->policy_x, c->policy_q, c->small_recs, c->small_out, c->small_args,
                   c->grid_partials, c->grid_bar, c->pow_ticket};
    for (void *p : dev)
        if (p) cudaFree(p);
    free_tiles(c->TX);
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
    a.wstart = d.wstart; a.nruns = d.nruns; a.col = d.col; a.cols = d.cols; a.skip = skip;
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
    e.c32 = c->cp32; e.c32lo = c->cp32lo; e.l32 = c->lp32; e.u32 = c->up32; e.x032 = c->x032;
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
    e.b32 = c->bp32; e.b32lo = c->bp32lo; e.y032 = c->y032;
    e.ctl = c->ctl; e.it = it; e.ineq = c->ineq; e.reflect = (int)c->opt.reflect;
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

// the two phases of a normal iteration, as a solve launches them (programmatic dependent
// launches)
// the x phase of a normal FP64 iteration on the gather-tiled layout: k_tile_part (y in
// shared memory, partial sums) then k_tile_epi (the sums and the x update), both launched
// as programmatic dependents like the sliced-ELL phases
int launch_tiles_x(hpr_ctx *ctx, int it)
{
    const TileDev &T = ctx->TX;
    TileArgs a{};
    a.cta_blk = T.cta_blk; a.bstart = T.bstart; a.ustart = T.ustart; a.wstart = T.wstart;
    a.smeta = T.smeta; a.oslot = T.oslot; a.val = T.val; a.col = T.col;
    a.P = T.P; a.ctr = T.ctr; a.g = ctx->y;
    a.trigger_from = 0;                          // one CTA per SM: a single wave
    TileEpiArgs b{};
    b.rows = (int)ctx->n; b.nblk = T.nblk; b.slot_ptr = T.slot_ptr; b.P = T.P; b.ctr = T.ctr;
    const int ge = (int)((ctx->n + TB - 1) / TB);
    b.trigger_from = std::max(0, ge - (2048 / TB) * ctx->num_sms);
    const EpiX<false> e = epi_x<false>(ctx, it);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg{};
    cfg.stream = ctx->stream;
    cfg.attrs = attr;
    cfg.numAttrs = ctx->opt.pdl ? 1 : 0;
    cfg.gridDim = dim3((unsigned)T.grid);
    cfg.blockDim = dim3(TILE_TB);
    cfg.dynamicSmemBytes = sizeof(double) * (size_t)T.glen_max;
    CK(cudaLaunchKernelEx(&cfg, k_tile_part, a));
    cfg.gridDim = dim3((unsigned)ge);
    cfg.blockDim = dim3(TB);
    cfg.dynamicSmemBytes = 0;
    CK(cudaLaunchKernelEx(&cfg, k_tile_epi<EpiX<false>>, b, e));
    ctx->launches += 2;
    return HPR_OK;
}

bool tiles_on(const hpr_ctx *ctx) { return ctx->TX.nblk > 0 && ctx->opt.gather_tiles != 0; }

int launch_normal_x(hpr_ctx *ctx, int it)
{
    if (ctx->form == 1) return launch_sell_pdl(ctx, ctx->ST, epi_x32<false>(ctx, it));
    if (tiles_on(ctx)) return launch_tiles_x(ctx, it);
    return launch_sell_pdl(ctx, ctx->ST, epi_x<false>(ctx, it));
}

int launch_normal_y(hpr_ctx *ctx, int it)
{
    if (ctx->form == 1) return launch_sell_pdl(ctx, ctx->SA, epi_y32<false>(ctx, it));
    return launch_sell_pdl(ctx, ctx->SA, epi_y<false>(ctx, it));
}

// one HPR iteration (phase X then phase Y).  store: the phases also store x_bar, z_bar,
// y_bar, x - x_bar, y - y_bar; check: the two residual passes run and every check
// quantity is reduced into scal slot `slot`.
int enqueue_iteration(hpr_ctx *ctx, int it, bool store, bool check, int slot)
{
    int st;
    if (ctx->form == 1 && (store || check)) {
        if ((st = launch_sell(ctx, ctx->ST, epi_x32<true>(ctx, it)))) return st;
        if ((st = launch_sell(ctx, ctx->SA, epi_y32<true>(ctx, it)))) return st;
    } else if (store || check) {
        if ((st = launch_sell(ctx, ctx->ST, epi_x<true>(ctx, it)))) return st;
        if ((st = launch_sell(ctx, ctx->SA, epi_y<true>(ctx, it)))) return st;
    } else {
        if ((st = launch_normal_x(ctx, it))) return st;
        if ((st = launch_normal_y(ctx, it))) return st;
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
    CKA(cudaMalloc((void **)&ctx->ctl, ctx->ctl_bytes));
    CKA(cudaMallocHost((void **)&ctx->ctl_h, ctx->ctl_bytes));
    memset(ctx->ctl_h, 0, ctx->ctl_bytes);
    ctx->ctl_cap = cap;
    return HPR_OK;
}

// ---------------------------------------------------------------- power method

double small_fp64_per_iter(const hpr_ctx *ctx);
constexpr double SMALL_POWER_FP64_MAX = 600.0;
constexpr size_t SMALL_POWER_SMEM_MAX = 200 * 1024;

// the power method in one CTA (k_power_small) when the LP fits one SM and its FP64 work per
// step is small: the same steps as the multi-CTA kernels, two block barriers a step instead
// of two launches
int run_power_small(hpr_ctx *ctx, bool *done)
{
    *done = false;
    const size_t smem = sizeof(double) * (size_t)(ctx->m + ctx->n);
    if (smem > SMALL_POWER_SMEM_MAX || small_fp64_per_iter(ctx) > SMALL_POWER_FP64_MAX) return HPR_OK;
    hprsmall::SmallArgs A{};
    auto mat_of = [](const SellDev &D) {
        hprsmall::SmallMat M{};
        M.nslices = D.nslices; M.cols = D.cols; M.entries = D.entries;
        M.srow = D.srow; M.sptr = D.sptr; M.col = D.col; M.slg = D.slg; M.val = D.val;
        return M;
    };
    A.m = (int)ctx->m; A.n = (int)ctx->n;
    A.A = mat_of(ctx->SA); A.T = mat_of(ctx->ST);
    A.seed = ctx->opt.seed; A.perm_r = ctx->perm_r;
    A.power_tol = ctx->opt.power_tol;
    A.power_max_iter = std::max<int64_t>(1, ctx->opt.power_max_iter);
    if (!ctx->small_args) DALLOC(ctx->small_args, 1);
    if (!ctx->small_out) DALLOC(ctx->small_out, hprsmall::SO_LEN);
    CK(cudaMemcpyAsync(ctx->small_args, &A, sizeof A, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaFuncSetAttribute(hprsmall::k_power_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    hprsmall::k_power_small<<<1, hprsmall::NT, smem, ctx->stream>>>(ctx->small_args, ctx->small_out);
    CKL();
    ctx->launches += 1;
    double h[3];
    CK(cudaMemcpyAsync(h, ctx->small_out, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->lambda = h[0];
    ctx->power_iters = (int64_t)h[1];
    ctx->power_rel_change = h[2];
    if (!std::isfinite(ctx->lambda) || !(ctx->lambda > 0.0))
        return fail_arg(ctx, HPR_ERR_NUMERIC, "power method returned a non-positive lambda");
    *done = true;
    return HPR_OK;
}

int run_power(hpr_ctx *ctx)
{
    {
        bool done = false;
        int r = run_power_small(ctx, &done);
        if (r || done) return r;
    }
    const int64_t m = ctx->m;
    const int gm = (int)((m + TB - 1) / TB);
    // tickets of the two launches: a group counter per POW_GROUP CTAs and one over the groups
    const int64_t tstride = 1 + ((int64_t)ctx->pstride + POW_GROUP - 1) / POW_GROUP;
    if (ctx->pow_ticket_len < 2 * tstride) {
        if (ctx->pow_graph) cudaGraphExecDestroy(ctx->pow_graph);
        ctx->pow_graph = nullptr;
        if (ctx->pow_ticket) cudaFree(ctx->pow_ticket);
        ctx->pow_ticket = nullptr;
        ctx->pow_ticket_len = 0;
        DALLOC(ctx->pow_ticket, 2 * tstride);
        CK(cudaMemsetAsync(ctx->pow_ticket, 0, sizeof(unsigned) * 2 * tstride, ctx->stream));
        ctx->pow_ticket_len = 2 * tstride;
    }
    // w (m) in dy: the start vector, then A s; s = A^T w / ||w|| (n) in dx
    double *u = ctx->dy, *s = ctx->dx;
    k_pow_start<<<gm, TB, 0, ctx->stream>>>((int)m, ctx->opt.seed, ctx->perm_r, u, ctx->partials,
                                             ctx->pstride);
    CKL();
    int st = launch_reduce(ctx, {{Q_V2, gm}}, ctx->scal);
    if (st) return st;
    PowCtl pc{};
    pc.tol = ctx->opt.power_tol;
    pc.max_iter = (int)std::max<int64_t>(1, ctx->opt.power_max_iter);
    *ctx->pctl_h = pc;
    CK(cudaMemcpyAsync(ctx->pctl, ctx->pctl_h, sizeof(PowCtl), cudaMemcpyHostToDevice, ctx->stream));
    // the first step normalises the start vector inside its row sums: inv = 1 / ||w||
    k_inv_sqrt_scalar<<<1, 1, 0, ctx->stream>>>(ctx->scal, Q_V2, &ctx->pctl->inv);
    CKL();

    // two launches a step (EpiPowT, EpiPowA): each folds the previous normalisation or
    // reduction into its own row sums / last CTA
    EpiPowT et{};
    et.xa = et.xb = u; et.q[0] = Q_S2; et.partials = ctx->partials; et.pstride = ctx->pstride; et.out = s;
    et.pc = ctx->pctl;
    EpiPowA ea{};
    ea.xa = ea.xb = s; ea.q[0] = Q_W2; ea.partials = ctx->partials; ea.pstride = ctx->pstride; ea.out = u;
    ea.pc = ctx->pctl;
    auto launch_pow = [&](const SellDev &M, auto e, unsigned *ticket) -> int {
        if (M.rows == 0) return HPR_OK;
        k_sell_pow<<<M.grid, SELL_TB, 0, ctx->stream>>>(sell_of(M, false, &ctx->pctl->done), e, ticket);
        CKL();
        ctx->launches += 1;
        return HPR_OK;
    };
    auto enqueue_steps = [&](int steps) -> int {
        for (int k = 0; k < steps; ++k) {
            int r = launch_pow(ctx->ST, et, ctx->pow_ticket);
            if (r) return r;
            r = launch_pow(ctx->SA, ea, ctx->pow_ticket + tstride);
            if (r) return r;
        }
        return HPR_OK;
    };

    const int BATCH = 16;
    if (ctx->opt.use_graph && !ctx->pow_graph) {
        cudaGraph_t g;
        CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        const int64_t before = ctx->launches;
        int r = enqueue_steps(BATCH);
        ctx->pow_graph_launches = ctx->launches - before;
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
    ctx->launches += 2;   // start vector, 1/norm (+1 for the reduction above)
    for (int64_t done_steps = 0; done_steps <= ctx->opt.power_max_iter; done_steps += BATCH) {
        if (ctx->opt.use_graph) {
            ctx->launches += ctx->pow_graph_launches;
            CK(cudaGraphLaunch(ctx->pow_graph, ctx->stream));
        } else {
            int r = enqueue_steps(BATCH);
            if (r) return r;
        }
        CK(cudaMemcpyAsync(ctx->pctl_h, ctx->pctl, sizeof(PowCtl), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        if (ctx->pctl_h->done) break;
    }
    ctx->lambda = ctx->pctl_h->lam;
    ctx->power_iters = ctx->pctl_h->k;
    ctx->power_rel_change = ctx->pctl_h->rel_change;
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
    D.cols = (&D == &ctx->ST) ? (int)ctx->m : (int)ctx->n;
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
        k_gather_src<<<grid_for(D.entries), 256, 0, s>>>(D.entries, csr_val, (int)ctx->nnz, D.src, D.val); CKL();
        k_narrow<<<grid_for(D.entries), 256, 0, s>>>(D.entries, D.val, D.val32); CKL();
    }
    CK(cudaStreamSynchronize(s));
    return HPR_OK;
}

// device copy of a gather-tiled layout (values gathered later from the scaled CSR values
// through `src`, see tile_values)
int upload_tiles(hpr_ctx *ctx, TileDev &T, const TileHost &H, int rows)
{
    cudaStream_t s = ctx->stream;
    T.nblk = H.nblk;
    T.grid = (int)H.cta_blk.size();
    T.glen_max = H.glen_max;
    T.entries = (int64_t)H.col.size();
    T.nsub = (int64_t)H.oslot.size();
    auto up = [&](auto *&d, const auto &v) -> int {
        using E = typename std::remove_reference<decltype(v)>::type::value_type;
        DALLOC(d, (int64_t)std::max<size_t>(v.size(), 1));
        if (!v.empty()) CK(cudaMemcpyAsync(d, v.data(), sizeof(E) * v.size(), cudaMemcpyHostToDevice, s));
        return HPR_OK;
    };
    int st;
    if ((st = up(T.cta_blk, H.cta_blk)) || (st = up(T.bstart, H.bstart)) || (st = up(T.ustart, H.ustart)) ||
        (st = up(T.wstart, H.wstart)) || (st = up(T.smeta, H.smeta)) ||
        (st = up(T.oslot, H.oslot)) || (st = up(T.slot_ptr, H.slot_ptr)) || (st = up(T.src, H.src)) ||
        (st = up(T.col, H.col)))
        return st;
    DALLOC(T.val, std::max<int64_t>(T.entries, 1));
    DALLOC(T.P, std::max<int64_t>(T.nsub, 1));
    DALLOC(T.ctr, T.nblk);
    CK(cudaMemsetAsync(T.ctr, 0, sizeof(unsigned) * T.nblk, s));
    (void)rows;
    return HPR_OK;
}

// the tiled layout's values from the scaled CSR values of A^T
int tile_values(hpr_ctx *ctx, TileDev &T)
{
    if (!T.nblk || !T.entries) return HPR_OK;
    k_gather_src<<<grid_for(T.entries), 256, 0, ctx->stream>>>(T.entries, ctx->T_val, (int)ctx->nnz, T.src, T.val);
    CKL();
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
    // the gather-tiled x phase (k_tile_part): y in blocks of shared memory
    TileHost hX;
    bool tiles = false;
    if (op.gather_tiles != 0) {
        int smem = 0;
        CK(cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
        const int cap = std::min(65536, (smem - 1024) / 8) & ~1;
        const int len = op.tile_len > 0 ? (int)std::min<int64_t>(op.tile_len, cap) : cap;
        // option 1: a phase that moves enough data to be bound by its gathers, with at least
        // 4 CTAs per block of y
        const bool want = op.gather_tiles == 2 ||
                          (!smallT && (m + len - 1) / len <= ctx->num_sms / 4);
        if (want) tiles = build_tiles(trp, tci, (int)n, pc, ipr, (int)m, len, ctx->num_sms, stepsT, costT, hX);
        if (!tiles && op.gather_tiles == 2)
            return fail_arg(ctx, HPR_ERR_ARG, "gather_tiles = 2: y needs more blocks than the GPU has SMs, "
                                              "or the layout's offsets exceed 32 bits");
    }
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
        D.cols = (&D == &ctx->ST) ? (int)ctx->m : (int)ctx->n;
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
    if (tiles) {
        if ((st0 = upload_tiles(ctx, ctx->TX, hX, (int)n))) return st0;
        CK(cudaFuncSetAttribute(k_tile_part, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(double) * ctx->TX.glen_max));
    }
    DALLOC(ctx->perm_r, m); DALLOC(ctx->perm_c, n); DALLOC(ctx->ineq, m);

    DALLOC(ctx->bp, m); DALLOC(ctx->wrp, m); DALLOC(ctx->cp, n); DALLOC(ctx->lp, n); DALLOC(ctx->up, n);
    DALLOC(ctx->wcp, n); DALLOC(ctx->unperm, n + m);
    DALLOC(ctx->x32, n); DALLOC(ctx->xhat32, n); DALLOC(ctx->y32, m);
    DALLOC(ctx->x032, n); DALLOC(ctx->y032, m);
    DALLOC(ctx->cp32, n); DALLOC(ctx->lp32, n); DALLOC(ctx->up32, n); DALLOC(ctx->bp32, m);
    DALLOC(ctx->cp32lo, n); DALLOC(ctx->bp32lo, m);
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
    CKA(cudaMallocHost((void **)&ctx->scal_h, sizeof(double) * 2 * NQ));
    CKA(cudaMallocHost((void **)&ctx->pctl_h, sizeof(PowCtl)));
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
        k_scale_rows_cols<<<gm, 256, 0, s>>>((int)m, (int)n, ctx->A_rp, ctx->A_ci, ctx->A_val, dr, dc); CKL();
    }
    if (ctx->opt.pc_alpha >= 0.0) {
        const double al = ctx->opt.pc_alpha;
        k_gather<<<gz, 256, 0, s>>>(nnz, ctx->A_val, ctx->T_perm, ctx->T_val); CKL();
        k_row_abspow<<<gm, 256, 0, s>>>((int)m, ctx->A_rp, ctx->A_val, 2.0 - al, dr); CKL();
        k_row_abspow<<<gn, 256, 0, s>>>((int)n, ctx->T_rp, ctx->T_val, al, dc); CKL();
        k_factor<<<gm, 256, 0, s>>>((int)m, dr, ctx->Dr); CKL();
        k_factor<<<gn, 256, 0, s>>>((int)n, dc, ctx->Dc); CKL();
        k_scale_rows_cols<<<gm, 256, 0, s>>>((int)m, (int)n, ctx->A_rp, ctx->A_ci, ctx->A_val, dr, dc); CKL();
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
    k_gather_src<<<grid_for(ctx->SA.entries), 256, 0, s>>>(ctx->SA.entries, ctx->A_val, (int)ctx->nnz, ctx->SA.src, ctx->SA.val); CKL();
    k_gather_src<<<grid_for(ctx->ST.entries), 256, 0, s>>>(ctx->ST.entries, ctx->T_val, (int)ctx->nnz, ctx->ST.src, ctx->ST.val); CKL();
    if ((st = tile_values(ctx, ctx->TX))) return st;
    k_narrow<<<grid_for(ctx->SA.entries), 256, 0, s>>>(ctx->SA.entries, ctx->SA.val, ctx->SA.val32); CKL();
    k_narrow<<<grid_for(ctx->ST.entries), 256, 0, s>>>(ctx->ST.entries, ctx->ST.val, ctx->ST.val32); CKL();
    k_permute<<<gm, 256, 0, s>>>(m, ctx->b_s, ctx->perm_r, ctx->bp); CKL();
    k_permute<<<gm, 256, 0, s>>>(m, ctx->wr, ctx->perm_r, ctx->wrp); CKL();
    k_permute<<<gn, 256, 0, s>>>(n, ctx->c_s, ctx->perm_c, ctx->cp); CKL();
    k_permute<<<gn, 256, 0, s>>>(n, ctx->l_s, ctx->perm_c, ctx->lp); CKL();
    k_permute<<<gn, 256, 0, s>>>(n, ctx->u_s, ctx->perm_c, ctx->up); CKL();
    k_permute<<<gn, 256, 0, s>>>(n, ctx->wc, ctx->perm_c, ctx->wcp); CKL();
    // FP32 copies of the data for the FP32 form's normal iterations (infinite bounds stay infinite)
    k_split32<<<gn, 256, 0, s>>>(n, ctx->cp, ctx->cp32, ctx->cp32lo); CKL();
    k_narrow<<<gn, 256, 0, s>>>(n, ctx->lp, ctx->lp32); CKL();
    k_narrow<<<gn, 256, 0, s>>>(n, ctx->up, ctx->up32); CKL();
    k_split32<<<gm, 256, 0, s>>>(m, ctx->bp, ctx->bp32, ctx->bp32lo); CKL();
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
    o->gather_tiles = 0;
    o->tile_len = 0;
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
    if (o->persistent < 0 || o->persistent > 4) return fail_arg(ctx, HPR_ERR_ARG, "persistent must be 0, 1, 2, 3 or 4");
    if (o->pdl != 0 && o->pdl != 1) return fail_arg(ctx, HPR_ERR_ARG, "pdl must be 0 or 1");
    if (o->gather_tiles < 0 || o->gather_tiles > 2) return fail_arg(ctx, HPR_ERR_ARG, "gather_tiles must be 0, 1 or 2");
    if (o->tile_len < 0 || o->tile_len == 1 || o->tile_len > 65536)
        return fail_arg(ctx, HPR_ERR_ARG, "tile_len must be 0 or in [2, 65536]");
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
    for (auto &kv : {std::make_pair("HPR_FAULT_ALLOC", &ctx->fault_alloc),
                     std::make_pair("HPR_FAULT_NAN_CHECK", &ctx->fault_nan_check),
                     std::make_pair("HPR_FAULT_BARRIER", &ctx->fault_barrier),
                     std::make_pair("HPR_GRID_CTAS", &ctx->grid_ctas_env)}) {
        const char *v = std::getenv(kv.first);
        *kv.second = v ? std::max(0LL, std::atoll(v)) : 0;
    }
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
    if (opt->reflect != ctx->opt.reflect || (opt->gather_tiles != 0) != (ctx->opt.gather_tiles != 0)) {
        // captured graphs hold the kernels and their arguments
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

#include "hpr_api_solve.cuh"
#include "hpr_api_batch.cuh"
#include "hpr_api_policy.cuh"
#include "hpr_api_noalloc.cuh"
#include "hpr_api_probe.cuh"
