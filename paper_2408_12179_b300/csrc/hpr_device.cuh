// Device code of the B300 HPR-LP solver (sm_103a).
//
// The hot path is the HPR iteration of Algorithm 2 with the closed forms of
// Section 3.3 (eq. update-x, update-y-2) and the reflection / Halpern steps:
//
//   phase X (over the rows of A^T, i.e. the columns j of A):
//       s = (A^T y)_j;  v = x_j + sigma (s - c_j);  xbar = Pi_[l_j,u_j](v)
//       xhat_j = 2 xbar - x_j;  x_j <- x0_j/(t+2) + (t+1)/(t+2) xhat_j
//   phase Y (over the rows i of A):
//       q = (A xhat)_i;  ybar = y_i + (b_i - q)/(lambda sigma), clamped at 0 for i >= m1
//       yhat = 2 ybar - y_i;  y_i <- y0_i/(t+2) + (t+1)/(t+2) yhat
//
// Both phases are one sparse matrix-vector product each with the elementwise work
// fused as an epilogue, so every vector crosses HBM once per iteration.  B300 executes
// FP64 at a small fraction of its FP32 rate, so the products use a sliced-ELL layout in
// which every FP64 instruction is issued by a full warp of useful lanes (see k_sell).
// All reductions (row sums, CTA partials, final sums) have a fixed order, so results
// are bitwise reproducible.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace hprdev {

// ---- bounds-checking build (HPR_BOUNDS_CHECK): every gather's index is checked against
// the gathered vector's length before the load; an index out of range is counted in a
// device counter (read with hpr_bounds_violations) and replaced by 0, so that the load
// stays in bounds and the kernel runs on (no trap).  In the normal build HPR_COL is the
// index itself.
#ifdef HPR_BOUNDS_CHECK
__device__ unsigned long long g_bounds_violations = 0;
__device__ __forceinline__ int col_checked(int c, int len)
{
    if ((unsigned)c >= (unsigned)len) {
        atomicAdd(&g_bounds_violations, 1ull);
        return 0;
    }
    return c;
}
#define HPR_COL(c, len) ::hprdev::col_checked((c), (len))
#else
#define HPR_COL(c, len) (c)
#endif

constexpr int TB = 256;                 // threads per CTA (vector, reduction kernels)
#ifndef HPR_SELL_TB
#define HPR_SELL_TB 64
#endif
#ifndef HPR_SELL_CTAS
#define HPR_SELL_CTAS 16
#endif
// The sliced-ELL kernels run small CTAs: one work unit per warp, 2 warps per CTA, so the
// hardware block scheduler balances the units' uneven costs at a fine grain and a CTA
// whose warps finish early frees its slot at once.
constexpr int SELL_TB = HPR_SELL_TB;             // threads per sliced-ELL CTA
constexpr int SELL_WARPS = SELL_TB / 32;         // work units per sliced-ELL CTA
constexpr int SELL_CTAS_PER_SM = HPR_SELL_CTAS;  // resident CTAs of the sliced-ELL kernels

// quantities reduced at a check (indices into the partials / scalar arrays)
enum {
    Q_DX2 = 0,   // ||x - xbar||^2                      (phase X, check mode)
    Q_XX0 = 1,   // ||xbar - x0||^2
    Q_CX = 2,    // <c_s, xbar>
    Q_BND = 3,   // sum_{z>0} z l_s + sum_{z<0} z u_s
    Q_DY2 = 4,   // ||y - ybar||^2                      (phase Y, check mode)
    Q_YY0 = 5,   // ||ybar - y0||^2
    Q_BY = 6,    // <b_s, ybar>
    Q_RD = 7,    // ||w_c (c_s - A^T ybar - zbar)||^2   (dual residual pass)
    Q_RP = 8,    // ||w_r Pi_D(b_s - A xbar)||^2        (primal residual pass)
    Q_CROSS = 9, // <y - ybar, A (x - xbar)>
    Q_S2 = 10,   // power method: ||A^T u||^2
    Q_W2 = 11,   // power method: ||A A^T u||^2
    Q_V2 = 12,   // generic vector norm (start vector, b, c)
    Q_V2B = 13,
    Q_POWG = 14, // power method: group sums of the CTA partials
    NQ = 16
};

// Per-period control block written by the host before each check period.
struct DevCtl {
    double sigma;     // sigma_r
    double inv_ls;    // 1 / (lambda sigma_r)
    int fused_lo, fused_hi;   // iterations [fused_lo, fused_hi) of the period that fused
                              // (batched) launches run for this context
    int form;         // 0: FP64 iterates, 1: FP32 form
    int active;       // 0: the context's solve has ended (fused launches skip it)
    int check_a, check_b;     // the period's check-mode iterations (-1: none): its first
                              // (an inner loop starts) and its last
    double pad[3];
    double h[2];      // h[2i] = 1/(t+2), h[2i+1] = (t+1)/(t+2) for iteration i of the period
};

struct PowCtl {
    double lam, lam_prev, inv, tol;
    int k, done, max_iter, stop_after;
    double rel_change;    // |lambda_k - lambda_{k-1}| / lambda_k of the last step (k > 1)
};

// ------------------------------------------------------------------ block reduction
// Fixed-order sum of one double per thread over an NT-thread block; result valid in
// thread 0.  Order: xor-butterfly inside each warp, then the NT/32 warp sums in order.
template <int NT = TB>
__device__ __forceinline__ double block_sum(double v, double *scratch /* >= NT/32 */)
{
    static_assert(NT % 32 == 0 && NT >= 32, "whole warps");
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) scratch[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        s = scratch[0];
#pragma unroll
        for (int i = 1; i < NT / 32; ++i) s += scratch[i];
    }
    return s;
}

// ------------------------------------------------------------------ FP64-free helpers
// Order-preserving map of a (non-NaN) double onto a signed 64-bit integer, so that the
// projections compare on the integer pipes (B300's FP64 pipe is the scarce one).
__device__ __forceinline__ long long dkey(double v)
{
    const long long i = __double_as_longlong(v);
    return i ^ ((i >> 63) & 0x7fffffffffffffffLL);
}

// min(max(v, l), u) for l <= u (Pi_[l,u]); -0 orders below +0
__device__ __forceinline__ double clamp_lu(double v, double l, double u)
{
    const long long kv = dkey(v);
    double r = v;
    if (kv < dkey(l)) r = l;
    if (kv > dkey(u)) r = u;
    return r;
}

// max(v, 0) (Pi_{R_+}) from the sign bit
__device__ __forceinline__ double pos_part(double v)
{
    return __double_as_longlong(v) < 0 ? 0.0 : v;
}

// ------------------------------------------------------------------ sliced-ELL SpMV
// B300 issues one FP64 warp instruction every ~17 cycles per SM whatever the number of
// active lanes, and a dependent DFMA takes ~70 cycles.  So the SpMV keeps all 32 lanes
// of every FP64 instruction busy with useful work.  Rows are renumbered by decreasing
// length (stable) and taken in groups of 32.  A group gives each row L = 1, 2, ..., 32
// lanes (L grows with the group's longest row so that a slice needs at most ~40 steps)
// and is stored as L slices of 32/L rows, each column-major so that a warp reads 32
// consecutive values per step (sliced ELL with a global sort; padding entries are
// zeros).  A lane accumulates every L-th entry of its row with FMA; the L partial sums
// of a row are added by a fixed xor butterfly and moved to the row's own lane, so the
// epilogue of the group runs once, on 32 lanes, whatever L is.  The work units are light
// groups (whole) and the slices of heavy groups, longest first; each warp of the grid
// takes one unit, so the hardware's CTA scheduler balances the load.
// Row accumulators.  Acc<double>: FP64 FMA.  Acc<float> (the FP32 form): the FP32 product
// a*b is split exactly into p + e (e = fma(a, b, -p)) and accumulated in double-float
// (hi, lo) with Knuth's TwoSum, so a row sum of FP32 products keeps ~48 bits without a
// single FP64 instruction; the row's value is hi + lo in FP64.  Explicit round-to-nearest
// intrinsics keep the compiler from contracting the error-free transformations.
template <class V>
struct Acc;

template <>
struct Acc<double> {
    double a = 0.0;
    __device__ __forceinline__ void add(double v, double g) { a = fma(v, g, a); }
    __device__ __forceinline__ void merge(const Acc &o) { a += o.a; }
    __device__ __forceinline__ void xor_reduce(int o) { a += __shfl_xor_sync(0xffffffffu, a, o); }
    __device__ __forceinline__ double value() const { return a; }
    template <class S>
    __device__ __forceinline__ S value_as() const { return a; }
};

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

template <>
struct Acc<float> {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add(float v, float g)
    {
        const float p = __fmul_rn(v, g);
        const float pe = __fmaf_rn(v, g, -p);     // exact: v*g = p + pe
        float s, e;
        two_sum(hi, p, s, e);
        hi = s;
        lo = __fadd_rn(lo, __fadd_rn(e, pe));
    }
    __device__ __forceinline__ void merge(const Acc &o)
    {
        float s, e;
        two_sum(hi, o.hi, s, e);
        hi = s;
        lo = __fadd_rn(lo, __fadd_rn(e, o.lo));
    }
    __device__ __forceinline__ void xor_reduce(int o)
    {
        Acc t;
        t.hi = __shfl_xor_sync(0xffffffffu, hi, o);
        t.lo = __shfl_xor_sync(0xffffffffu, lo, o);
        merge(t);
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
    // the row sum as a normalised double-float pair (the FP32 form's normal iterations, which
    // issue no FP64 instruction), or as FP64
    template <class S>
    __device__ __forceinline__ S value_as() const
    {
        if constexpr (sizeof(S) == 8 && !std::is_same<S, double>::value) {
            float h, l;
            two_sum(hi, lo, h, l);
            return S{h, l};
        } else {
            return value();
        }
    }
};

// a - b of two double-float values (a_hi + a_lo, b_hi + b_lo), rounded once to FP32: the
// difference keeps FP32 precision relative to ITSELF even when a and b nearly cancel
__device__ __forceinline__ float df_sub(float ah, float al, float bh, float bl)
{
    float d, e;
    two_sum(ah, -bh, d, e);
    return __fadd_rn(d, __fadd_rn(e, __fsub_rn(al, bl)));
}

struct SellArgs {
    int rows;             // rows of the matrix (in the renumbered order)
    int nslices;
    const int *srow;      // nslices + 1: first row of each slice
    const int *sptr;      // nslices + 1: first stored entry; slice s has (sptr[s+1]-sptr[s])/32 steps
    const unsigned char *slg;   // log2 of the lanes per row of each slice
    int nruns;            // work units, one per warp
    const int *wstart;    // nruns + 1: unit i covers slices [wstart[i], wstart[i+1])
    const void *val;      // stored values, double or float (E::Val); padding: 0
    const int *col;       // stored column indices (padding: 0)
    int cols;             // length of the gathered vectors (columns of the matrix)
    const int *skip;      // optional: the kernel does nothing while *skip != 0
    int trigger_from;     // programmatic launch: CTAs from this index on let the next kernel
                          // start once they have waited for the previous one (others: at exit)
};

// Programmatic dependent launch (the phases of a normal iteration are launched with it):
// the work before griddepcontrol.wait -- unit metadata and the epilogue operands, none of
// them written by the kernel just before -- overlaps that kernel's tail; both instructions
// are no-ops for a kernel launched without the attribute.
__device__ __forceinline__ void dep_wait_and_trigger(const SellArgs &S)
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if ((int)blockIdx.x >= S.trigger_from) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ double shfl_sum(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ float2 shfl_sum(float2 v, int src)
{
    return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// E supplies the value type Val (double or float) of the stored values and gathered
// vectors, NV gathered vectors xa (, xb), NP partial sums (ids q[]), a Pre record of
// epilogue operands (prefetch(j)) and row(j, act, s, pre, part) with FP64 row sums s.
template <class E>
__device__ __forceinline__ void sell_unit(const SellArgs &S, const E &ee, int run, double *part)
{
    constexpr int NV = E::NV;
    using V = typename E::Val;
    using Sm = typename E::Sum;                  // type of the row sums the epilogue takes
    const int lane = threadIdx.x & 31;
    bool waited = false;
    int buf_r0 = 0, buf_n = 0;                   // rows [buf_r0, buf_r0 + buf_n) hold sums
    Sm buf0{}, buf1{};                           // lane t: sum of row buf_r0 + t
    typename E::Pre pre{};
    const int s_beg = run < S.nruns ? S.wstart[run] : 0;
    const int s_end = run < S.nruns ? S.wstart[run + 1] : 0;
    for (int s = s_beg; s < s_end; ++s) {
        const int lg = S.slg[s];
        const int r0 = S.srow[s], nrows = S.srow[s + 1] - r0;
        const int base = S.sptr[s];
        const int steps = (S.sptr[s + 1] - base) >> 5;
        if (buf_n + nrows > 32) {                 // run started inside a group: flush early
            const int j = min(buf_r0 + lane, S.rows - 1);
            const Sm sums[2] = {buf0, buf1};
            ee.row(j, lane < buf_n, sums, pre, part);
            buf_n = 0;
        }
        if (buf_n == 0) {
            buf_r0 = r0;                          // operands of the next 32 rows, early
            pre = ee.prefetch(min(r0 + lane, S.rows - 1));
            if (!waited) {                        // the gathered vector is the previous kernel's output
                dep_wait_and_trigger(S);
                waited = true;
            }
        }
        const V *pv = static_cast<const V *>(S.val) + base + lane;
        const int *pc = S.col + base + lane;
        Acc<V> a0, a1, b0, b1;
        int k = 0;
        for (; k + 4 <= steps; k += 4) {
            V v[4], g0[4], g1[4];
            int c[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                v[u] = __ldcs(pv + (k + u) * 32);
                c[u] = HPR_COL(__ldcs(pc + (k + u) * 32), S.cols);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                g0[u] = __ldg(ee.xa + c[u]);
                if (NV == 2) g1[u] = __ldg(ee.xb + c[u]);
            }
            // two chains (even / odd steps) halve the dependent FMA latency
            a0.add(v[0], g0[0]);
            a1.add(v[1], g0[1]);
            a0.add(v[2], g0[2]);
            a1.add(v[3], g0[3]);
            if (NV == 2) {
                b0.add(v[0], g1[0]);
                b1.add(v[1], g1[1]);
                b0.add(v[2], g1[2]);
                b1.add(v[3], g1[3]);
            }
        }
        if (steps == 1) {                         // one step (most rows of A^T of a sparse LP)
            const V v = __ldcs(pv + k * 32);
            const int c = HPR_COL(__ldcs(pc + k * 32), S.cols);
            const V g0 = __ldg(ee.xa + c);
            if (NV == 2) {
                const V g1 = __ldg(ee.xb + c);
                b0.add(v, g1);
            }
            a0.add(v, g0);
        } else if (steps < 4) {                   // a short slice: its 2-3 steps as one batch
            const int rem = steps;                // warp-uniform
            V v[3], g0[3], g1[3];
            int c[3];
#pragma unroll
            for (int u = 0; u < 3; ++u) {
                v[u] = u < rem ? __ldcs(pv + (k + u) * 32) : V(0);
                c[u] = u < rem ? HPR_COL(__ldcs(pc + (k + u) * 32), S.cols) : 0;
            }
#pragma unroll
            for (int u = 0; u < 3; ++u) {
                g0[u] = u < rem ? __ldg(ee.xa + c[u]) : V(0);
                if (NV == 2) g1[u] = u < rem ? __ldg(ee.xb + c[u]) : V(0);
            }
#pragma unroll
            for (int u = 0; u < 3; ++u) {         // same order as step by step
                if (u < rem) {
                    a0.add(v[u], g0[u]);
                    if (NV == 2) b0.add(v[u], g1[u]);
                }
            }
        } else {
            for (; k < steps; ++k) {
                const V v = __ldcs(pv + k * 32);
                const int c = HPR_COL(__ldcs(pc + k * 32), S.cols);
                a0.add(v, __ldg(ee.xa + c));
                if (NV == 2) b0.add(v, __ldg(ee.xb + c));
            }
        }
        if (steps >= 4) {                         // warp-uniform
            a0.merge(a1);
            if (NV == 2) b0.merge(b1);
        }
        for (int o = 1; o < (1 << lg); o <<= 1) { // warp-uniform: lg is per slice
            a0.xor_reduce(o);
            if (NV == 2) b0.xor_reduce(o);
        }
        // row q of this slice (held by lanes q*L ...) moves to lane buf_n + q
        const int src = (int)(((unsigned)(lane - buf_n) << lg) & 31u);
        const Sm m0 = shfl_sum(a0.template value_as<Sm>(), src);
        const Sm m1 = NV == 2 ? shfl_sum(b0.template value_as<Sm>(), src) : Sm{};
        if (lane >= buf_n && lane < buf_n + nrows) {
            buf0 = m0;
            buf1 = m1;
        }
        buf_n += nrows;
        if (buf_n == 32 || s + 1 == s_end) {      // a full group (or the end of the run)
            const int j = min(buf_r0 + lane, S.rows - 1);
            const Sm sums[2] = {buf0, buf1};
            ee.row(j, lane < buf_n, sums, pre, part);
            buf_n = 0;
        }
    }
    if (!waited) dep_wait_and_trigger(S);        // warps without a work unit take part too
}

template <class E>
__global__ void __launch_bounds__(SELL_TB, SELL_CTAS_PER_SM) k_sell(SellArgs S, E e)
{
    constexpr int NP = E::NP;
    __shared__ double red[SELL_WARPS];
    if (S.skip && *S.skip) return;
    E ee = e;
    ee.load();
    const int run = blockIdx.x * SELL_WARPS + (threadIdx.x >> 5);   // one unit per warp
    double part[NP > 0 ? NP : 1];
#pragma unroll
    for (int i = 0; i < (NP > 0 ? NP : 1); ++i) part[i] = 0.0;
    sell_unit(S, ee, run, part);
    if (NP > 0) {
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            const double t = block_sum<SELL_TB>(part[i], red);
            if (threadIdx.x == 0) ee.partials[ee.q[i] * ee.pstride + blockIdx.x] = t;
        }
    }
}

// Many LPs in one launch (the batched solve).  Block b of a fused launch is CTA
// tasks[b].cta of context tasks[b].inst: its SELL_WARPS warps take that context's work
// units SELL_WARPS cta + w, exactly as block `cta` of the context's own launch would, so the
// per-row arithmetic and the per-CTA partial sums are the same.  The context's layout
// and epilogue operands come from per-context tables.  A whole block skips unless its
// context is active, in the form FORM (-1: any), and iteration `it` is one this launch
// runs for it: MODE 0 (normal iterations) fused_lo <= it < fused_hi, MODE 1 (check-mode
// iterations and residual passes) it == check_a or it == check_b.
struct MultiTask {
    int inst, cta;
};

__device__ __forceinline__ bool multi_runs(const DevCtl *c, int mode, int form, int it)
{
    if (!c->active || (form >= 0 && c->form != form)) return false;
    return mode == 0 ? (it >= c->fused_lo && it < c->fused_hi) : (it == c->check_a || it == c->check_b);
}

template <class E, int MODE, int FORM>
__global__ void __launch_bounds__(SELL_TB, SELL_CTAS_PER_SM) k_sell_multi(const MultiTask *__restrict__ tasks,
                                                                  const SellArgs *__restrict__ sells,
                                                                  const E *__restrict__ epis, int it)
{
    constexpr int NP = E::NP;
    static_assert(MODE == 1 || NP == 0, "normal iterations have no partial sums");
    __shared__ double red[SELL_WARPS];
    const MultiTask t = tasks[blockIdx.x];
    E ee = epis[t.inst];
    if (!multi_runs(ee.ctl, MODE, FORM, it)) return;        // the whole block
    ee.it = it;
    ee.load();
    const SellArgs S = sells[t.inst];
    double part[NP > 0 ? NP : 1];
#pragma unroll
    for (int i = 0; i < (NP > 0 ? NP : 1); ++i) part[i] = 0.0;
    sell_unit(S, ee, t.cta * SELL_WARPS + (threadIdx.x >> 5), part);
    if (NP > 0) {
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            const double s = block_sum<SELL_TB>(part[i], red);
            if (threadIdx.x == 0) ee.partials[ee.q[i] * ee.pstride + t.cta] = s;
        }
    }
}

// the check reductions of many contexts: block b sums quantity q of context inst over its
// cnt CTA partials (the order of k_reduce) into out[slot * NQ + q], slot 1 at the check
// iteration ending the period, 0 at its first
struct RedTask {
    const double *partials;
    int pstride, q, cnt, pad;
    const DevCtl *ctl;
    double *out;
};

__global__ void __launch_bounds__(TB) k_reduce_multi(const RedTask *__restrict__ tasks, int it)
{
    __shared__ double red[TB / 32];
    const RedTask t = tasks[blockIdx.x];
    if (!multi_runs(t.ctl, 1, -1, it)) return;
    double s = 0.0;
    for (int g = threadIdx.x; g < t.cnt; g += TB) s += t.partials[t.q * t.pstride + g];
    s = block_sum(s, red);
    if (threadIdx.x == 0) t.out[(it == t.ctl->check_b ? NQ : 0) + t.q] = s;
}

// ------------------------------------------------------------------ epilogues
// phase X (rows of A^T = columns j of A): eq. (update-x), reflection, Halpern step;
// check mode also stores x_bar, z_bar (eq. update-z), x - x_bar and the partial sums
template <bool CHECK>
struct EpiX {
    using Val = double;
    using Sum = double;
    static constexpr int NV = 1, NP = CHECK ? 4 : 0;
    const double *xa, *xb;       // gathered: y
    int q[4];
    double *partials;
    int pstride;
    const double *c, *l, *u, *x0;
    double *x, *xhat, *xbar, *zbar, *dx;
    const DevCtl *ctl;           // sigma and the Halpern weights of iteration `it`
    int it;
    int reflect;                 // 1: Halpern target x_hat (Algorithm 2); 0: x_bar
    double sigma, ha, hb;
    struct Pre { double x, x0, c, l, u; };
    __device__ __forceinline__ void load()
    {
        sigma = ctl->sigma;
        ha = ctl->h[2 * it];
        hb = ctl->h[2 * it + 1];
    }
    __device__ __forceinline__ Pre prefetch(int j) const
    {
        return Pre{x[j], x0[j], c[j], l[j], u[j]};
    }
    __device__ __forceinline__ void row(int j, bool act, const double *s, const Pre &p,
                                        double *part) const
    {
        const double v = fma(sigma, s[0] - p.c, p.x);   // x + sigma (A^T y - c)
        const double xb_ = clamp_lu(v, p.l, p.u);       // Pi_C
        const double xh = fma(2.0, xb_, -p.x);          // 2 x_bar - x
        const double xn = fma(hb, reflect ? xh : xb_, ha * p.x0);   // x0/(t+2) + (t+1)/(t+2) x_hat
        if (act) {
            xhat[j] = xh;
            x[j] = xn;
        }
        if (CHECK && act) {
            const double zb = (xb_ - v) / sigma;
            const double d = p.x - xb_;
            xbar[j] = xb_;
            zbar[j] = zb;
            dx[j] = d;
            part[0] = fma(d, d, part[0]);
            part[1] = fma(xb_ - p.x0, xb_ - p.x0, part[1]);
            part[2] = fma(p.c, xb_, part[2]);
            if (zb > 0.0) part[3] = fma(zb, p.l, part[3]);
            else if (zb < 0.0) part[3] = fma(zb, p.u, part[3]);
        }
    }
};

// phase Y (rows i of A): eq. (update-y-2), reflection, Halpern step; check mode also
// stores y_bar, y - y_bar and the partial sums
template <bool CHECK>
struct EpiY {
    using Val = double;
    using Sum = double;
    static constexpr int NV = 1, NP = CHECK ? 3 : 0;
    const double *xa, *xb;       // gathered: x_hat
    int q[3];
    double *partials;
    int pstride;
    const double *b, *y0;
    double *y, *ybar, *dy;
    const DevCtl *ctl;           // 1/(lambda sigma) and the Halpern weights of iteration `it`
    int it;
    const unsigned char *ineq;   // ineq[i] = 1 for the rows of A2 (renumbered order)
    int reflect;                 // 1: Halpern target y_hat (Algorithm 2); 0: y_bar
    double inv_ls, ha, hb;
    struct Pre { double y, b, y0; unsigned char ineq; };
    __device__ __forceinline__ void load()
    {
        inv_ls = ctl->inv_ls;
        ha = ctl->h[2 * it];
        hb = ctl->h[2 * it + 1];
    }
    __device__ __forceinline__ Pre prefetch(int i) const
    {
        return Pre{y[i], b[i], y0[i], ineq[i]};
    }
    __device__ __forceinline__ void row(int i, bool act, const double *s, const Pre &p,
                                        double *part) const
    {
        double yb = fma(p.b - s[0], inv_ls, p.y);       // y + (b - A x_hat) / (lambda sigma)
        if (p.ineq) yb = pos_part(yb);                  // Pi_{R^m2_+}
        const double yh = fma(2.0, yb, -p.y);
        const double yn = fma(hb, reflect ? yh : yb, ha * p.y0);
        if (act) y[i] = yn;
        if (CHECK && act) {
            const double d = p.y - yb;
            ybar[i] = yb;
            dy[i] = d;
            part[0] = fma(d, d, part[0]);
            part[1] = fma(yb - p.y0, yb - p.y0, part[1]);
            part[2] = fma(p.b, yb, part[2]);
        }
    }
};

// The FP32 form (FP32 stored values and FP32 iterates x, x_hat, y): phase X.  Normal
// iterations run the update without a single FP64 instruction: the row sum arrives as the
// accumulators' double-float pair, c as a double-float pair of FP32 values, and s - c is
// formed by an error-free sum before it is rounded (the two nearly cancel near a solution:
// rounding them first would turn the difference into noise); l, u and the anchor x0 are FP32
// copies.  Check iterations (CHECK) take the FP64 row sum and FP64 data, as the FP64 form
// does, and store the FP64 x_bar, z_bar of the check.
template <bool CHECK>
struct EpiX32 {
    using Val = float;
    using Sum = typename std::conditional<CHECK, double, float2>::type;
    static constexpr int NV = 1, NP = CHECK ? 4 : 0;
    const float *xa, *xb;        // gathered: y (FP32)
    int q[4];
    double *partials;
    int pstride;
    const double *c, *l, *u, *x0;                 // FP64 data and anchor (checks)
    const float *c32, *c32lo, *l32, *u32, *x032;  // FP32 copies (normal iterations; c as hi + lo)
    float *x, *xhat;
    double *xbar, *zbar, *dx;
    const DevCtl *ctl;
    int it;
    int reflect;
    double sigma, ha, hb;
    float sigma32, ha32, hb32;
    struct PreC { double x0, c, l, u; float x; };
    struct PreF { float x0, ch, cl, l, u, x; };
    using Pre = typename std::conditional<CHECK, PreC, PreF>::type;
    __device__ __forceinline__ void load()
    {
        sigma = ctl->sigma;
        ha = ctl->h[2 * it];
        hb = ctl->h[2 * it + 1];
        sigma32 = (float)sigma;
        ha32 = (float)ha;
        hb32 = (float)hb;
    }
    __device__ __forceinline__ Pre prefetch(int j) const
    {
        if constexpr (CHECK) return Pre{x0[j], c[j], l[j], u[j], x[j]};
        else return Pre{x032[j], c32[j], c32lo[j], l32[j], u32[j], x[j]};
    }
    __device__ __forceinline__ void row(int j, bool act, const Sum *s, const Pre &p, double *part) const
    {
        if constexpr (!CHECK) {
            const float d = df_sub(s[0].x, s[0].y, p.ch, p.cl);             // A^T y - c
            const float v = __fmaf_rn(sigma32, d, p.x);
            const float xb_ = fminf(fmaxf(v, p.l), p.u);                    // Pi_C (l <= u)
            const float xh = __fmaf_rn(2.0f, xb_, -p.x);
            const float xn = __fmaf_rn(hb32, reflect ? xh : xb_, __fmul_rn(ha32, p.x0));
            if (act) {
                xhat[j] = xh;
                x[j] = xn;
            }
        } else {
            const double xj = (double)p.x;
            const double v = fma(sigma, s[0] - p.c, xj);
            const double xb_ = clamp_lu(v, p.l, p.u);
            const double xh = fma(2.0, xb_, -xj);
            const double xn = fma(hb, reflect ? xh : xb_, ha * p.x0);
            if (act) {
                xhat[j] = (float)xh;
                x[j] = (float)xn;
                const double zb = (xb_ - v) / sigma;
                const double dd = xj - xb_;
                xbar[j] = xb_;
                zbar[j] = zb;
                dx[j] = dd;
                part[0] = fma(dd, dd, part[0]);
                part[1] = fma(xb_ - p.x0, xb_ - p.x0, part[1]);
                part[2] = fma(p.c, xb_, part[2]);
                if (zb > 0.0) part[3] = fma(zb, p.l, part[3]);
                else if (zb < 0.0) part[3] = fma(zb, p.u, part[3]);
            }
        }
    }
};

// the FP32 form, phase Y (normal iterations: b - A x_hat by an error-free sum of double-float
// pairs, FP32 copies of y0)
template <bool CHECK>
struct EpiY32 {
    using Val = float;
    using Sum = typename std::conditional<CHECK, double, float2>::type;
    static constexpr int NV = 1, NP = CHECK ? 3 : 0;
    const float *xa, *xb;        // gathered: x_hat (FP32)
    int q[3];
    double *partials;
    int pstride;
    const double *b, *y0;
    const float *b32, *b32lo, *y032;
    float *y;
    double *ybar, *dy;
    const DevCtl *ctl;
    int it;
    const unsigned char *ineq;
    int reflect;
    double inv_ls, ha, hb;
    float inv_ls32, ha32, hb32;
    struct PreC { double b, y0; float y; unsigned char ineq; };
    struct PreF { float bh, bl, y0, y; unsigned char ineq; };
    using Pre = typename std::conditional<CHECK, PreC, PreF>::type;
    __device__ __forceinline__ void load()
    {
        inv_ls = ctl->inv_ls;
        ha = ctl->h[2 * it];
        hb = ctl->h[2 * it + 1];
        inv_ls32 = (float)inv_ls;
        ha32 = (float)ha;
        hb32 = (float)hb;
    }
    __device__ __forceinline__ Pre prefetch(int i) const
    {
        if constexpr (CHECK) return Pre{b[i], y0[i], y[i], ineq[i]};
        else return Pre{b32[i], b32lo[i], y032[i], y[i], ineq[i]};
    }
    __device__ __forceinline__ void row(int i, bool act, const Sum *s, const Pre &p, double *part) const
    {
        if constexpr (!CHECK) {
            const float d = df_sub(p.bh, p.bl, s[0].x, s[0].y);            // b - A x_hat
            float yb = __fmaf_rn(d, inv_ls32, p.y);
            if (p.ineq) yb = __float_as_int(yb) < 0 ? 0.0f : yb;          // Pi_{R_+}
            const float yh = __fmaf_rn(2.0f, yb, -p.y);
            if (act) y[i] = __fmaf_rn(hb32, reflect ? yh : yb, __fmul_rn(ha32, p.y0));
        } else {
            const double yi = (double)p.y;
            double yb = fma(p.b - s[0], inv_ls, yi);
            if (p.ineq) yb = pos_part(yb);
            const double yh = fma(2.0, yb, -yi);
            const double yn = fma(hb, reflect ? yh : yb, ha * p.y0);
            if (act) {
                y[i] = (float)yn;
                const double dd = yi - yb;
                ybar[i] = yb;
                dy[i] = dd;
                part[0] = fma(dd, dd, part[0]);
                part[1] = fma(yb - p.y0, yb - p.y0, part[1]);
                part[2] = fma(p.b, yb, part[2]);
            }
        }
    }
};

// hi + lo FP32 split of FP64 values: hi = fl32(v), lo = fl32(v - hi) (infinities: lo = 0)
__global__ void k_split32(int64_t len, const double *__restrict__ src, float *hi, float *lo)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = src[i];
        const float h = (float)v;
        hi[i] = h;
        lo[i] = isinf(v) ? 0.0f : (float)(v - (double)h);
    }
}

// dual residual of Section 4.1 in original-space weights w_c = beta_c / D_c
struct EpiDual {
    using Val = double;
    using Sum = double;
    static constexpr int NV = 1, NP = 1;
    const double *xa, *xb;       // gathered: y_bar
    int q[1];
    double *partials;
    int pstride;
    const double *c, *zbar, *wc;
    const DevCtl *ctl;           // batched launches only: whether this pass runs
    int it;
    struct Pre { double c, z, w; };
    __device__ __forceinline__ void load() {}
    __device__ __forceinline__ Pre prefetch(int j) const { return Pre{c[j], zbar[j], wc[j]}; }
    __device__ __forceinline__ void row(int, bool act, const double *s, const Pre &p, double *part) const
    {
        const double r = p.w * (p.c - s[0] - p.z);
        if (act) part[0] = fma(r, r, part[0]);
    }
};

// primal residual with weights w_r = beta_b / D_r and the cross term <dy, A dx> of the
// M-norm (eq. def:M with T1 = lambda I - A A^*)
struct EpiPrimal {
    using Val = double;
    using Sum = double;
    static constexpr int NV = 2, NP = 2;
    const double *xa, *xb;       // gathered: x_bar, x - x_bar
    int q[2];
    double *partials;
    int pstride;
    const double *b, *wr, *dy;
    const unsigned char *ineq;
    const DevCtl *ctl;           // batched launches only: whether this pass runs
    int it;
    struct Pre { double b, w, dy; unsigned char ineq; };
    __device__ __forceinline__ void load() {}
    __device__ __forceinline__ Pre prefetch(int i) const { return Pre{b[i], wr[i], dy[i], ineq[i]}; }
    __device__ __forceinline__ void row(int, bool act, const double *s, const Pre &p, double *part) const
    {
        double r = p.b - s[0];
        if (p.ineq) r = pos_part(r);                    // Pi_D
        r *= p.w;
        if (act) {
            part[0] = fma(r, r, part[0]);
            part[1] = fma(p.dy, s[1], part[1]);
        }
    }
};

// power method on A A^* (Section 4.1), two launches a step.  Step k: s = inv * A^T w (w is
// the previous step's A s, or the start vector, and inv its reciprocal norm, so the
// normalisation u = w / ||w|| rides in the row sums) with lambda_k = ||s||^2; then w = A s
// and inv = 1 / ||w||.  The last CTA of each launch to finish adds the CTA partial sums in
// a fixed order and takes the step's scalar decisions (convergence of lambda, the step
// cap, a zero w) on its thread 0.
struct EpiPowT {
    using Val = double;
    using Sum = double;
    static constexpr int NV = 1, NP = 1;
    const double *xa, *xb;       // gathered: w
    int q[1];
    double *partials;
    int pstride;
    double *out;                 // s
    PowCtl *pc;
    double inv;
    struct Pre { int unused; };
    __device__ __forceinline__ void load() { inv = pc->inv; }
    __device__ __forceinline__ Pre prefetch(int) const { return Pre{0}; }
    __device__ __forceinline__ void row(int j, bool act, const double *s, const Pre &, double *part) const
    {
        if (act) {
            const double t = s[0] * inv;
            out[j] = t;
            part[0] = fma(t, t, part[0]);
        }
    }
    // lambda_k = ||s||^2; stop when |lambda_k - lambda_{k-1}| <= tol lambda_k
    __device__ __forceinline__ void finish(double sum) const
    {
        pc->k += 1;
        pc->lam = sum;
        if (pc->k > 1) pc->rel_change = fabs(sum - pc->lam_prev) / sum;
        if (pc->k > 1 && fabs(sum - pc->lam_prev) <= pc->tol * sum) {
            pc->done = 1;
            return;
        }
        pc->lam_prev = sum;
        if (pc->k >= pc->max_iter) pc->stop_after = 1;
    }
};

struct EpiPowA {
    using Val = double;
    using Sum = double;
    static constexpr int NV = 1, NP = 1;
    const double *xa, *xb;       // gathered: s
    int q[1];
    double *partials;
    int pstride;
    double *out;                 // w
    PowCtl *pc;
    struct Pre { int unused; };
    __device__ __forceinline__ void load() {}
    __device__ __forceinline__ Pre prefetch(int) const { return Pre{0}; }
    __device__ __forceinline__ void row(int i, bool act, const double *s, const Pre &, double *part) const
    {
        if (act) {
            out[i] = s[0];
            part[0] = fma(s[0], s[0], part[0]);
        }
    }
    // inv = 1 / ||w|| for the next step (a zero w ends the method), and the step cap
    __device__ __forceinline__ void finish(double sum) const
    {
        const double nw = sqrt(sum);
        if (!(nw > 0.0)) {
            pc->done = 1;
            return;
        }
        pc->inv = 1.0 / nw;
        if (pc->stop_after) pc->done = 1;
    }
};

// A power-method launch: the phase kernel's row sums, then the CTA partial sums added in a
// fixed order, in two levels so that no CTA adds more than POW_GROUP of them: the last CTA
// of each group of POW_GROUP CTAs to finish adds its group's partials in CTA order, and the
// last group to finish adds the group sums in group order and calls finish.  ticket[0]
// counts the finished groups and ticket[1 + g] the finished CTAs of group g; the CTA that
// completes a counter resets it.
constexpr int POW_GROUP = 256;

template <class E>
__global__ void __launch_bounds__(SELL_TB, SELL_CTAS_PER_SM) k_sell_pow(SellArgs S, E e, unsigned *ticket)
{
    __shared__ double red[SELL_WARPS];
    __shared__ bool last;
    if (S.skip && *S.skip) return;
    E ee = e;
    ee.load();
    const int run = blockIdx.x * SELL_WARPS + (threadIdx.x >> 5);
    double part[1] = {0.0};
    sell_unit(S, ee, run, part);
    const double t = block_sum<SELL_TB>(part[0], red);
    const int G = (int)gridDim.x, grp = (int)blockIdx.x / POW_GROUP, ngrp = (G + POW_GROUP - 1) / POW_GROUP;
    const int g0 = grp * POW_GROUP, gsize = min(POW_GROUP, G - g0);
    double *const P = ee.partials + ee.q[0] * ee.pstride;
    double *const PG = ee.partials + Q_POWG * ee.pstride;
    if (threadIdx.x == 0) {
        P[blockIdx.x] = t;
        __threadfence();
        last = atomicAdd(ticket + 1 + grp, 1u) == (unsigned)gsize - 1u;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double sum = 0.0;
    for (int g = threadIdx.x; g < gsize; g += SELL_TB) sum += __ldcg(P + g0 + g);
    sum = block_sum<SELL_TB>(sum, red);
    if (threadIdx.x == 0) {
        ticket[1 + grp] = 0u;
        PG[grp] = sum;
        __threadfence();
        last = atomicAdd(ticket, 1u) == (unsigned)ngrp - 1u;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    sum = 0.0;
    for (int g = threadIdx.x; g < ngrp; g += SELL_TB) sum += __ldcg(PG + g);
    sum = block_sum<SELL_TB>(sum, red);
    if (threadIdx.x == 0) {
        ee.finish(sum);
        *ticket = 0u;
    }
}

// ------------------------------------------------------------------ final reduction
struct RedSpec {
    int nq;
    int q[NQ];
    int cnt[NQ];
};

// out[q] = sum of partials[q][0..cnt) in a fixed order (one CTA per quantity)
__global__ void __launch_bounds__(TB) k_reduce(const double *__restrict__ partials, int pstride,
                                               RedSpec spec, double *out, const int *skip)
{
    __shared__ double red[TB / 32];
    if (skip && *skip) return;
    const int q = spec.q[blockIdx.x], cnt = spec.cnt[blockIdx.x];
    double s = 0.0;
    for (int g = threadIdx.x; g < cnt; g += TB) s += partials[q * pstride + g];
    s = block_sum(s, red);
    if (threadIdx.x == 0) out[q] = s;
}

// ------------------------------------------------------------------ restart
// w^{r+1,0} = w_bar (Algorithm 2): x = x0 = xbar, y = y0 = ybar
__global__ void k_restart(int n, int m, const double *__restrict__ xbar,
                          const double *__restrict__ ybar, double *x, double *x0, double *y,
                          double *y0)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n + m; i += gridDim.x * blockDim.x) {
        if (i < n) {
            const double v = xbar[i];
            x[i] = v;
            x0[i] = v;
        } else {
            const double v = ybar[i - n];
            y[i - n] = v;
            y0[i - n] = v;
        }
    }
}

// restart in the FP32 form: x = (float) x_bar, x0 = x_bar and its FP32 copy, y likewise
__global__ void k_restart32(int n, int m, const double *__restrict__ xbar,
                            const double *__restrict__ ybar, float *x, double *x0, float *y,
                            double *y0, float *x032, float *y032)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n + m; i += gridDim.x * blockDim.x) {
        if (i < n) {
            const double v = xbar[i];
            x[i] = (float)v;
            x0[i] = v;
            x032[i] = (float)v;
        } else {
            const double v = ybar[i - n];
            y[i - n] = (float)v;
            y0[i - n] = v;
            y032[i - n] = (float)v;
        }
    }
}

// switch from the FP32 form to FP64 iterates: x = (double) x32, y = (double) y32
__global__ void k_widen(int n, int m, const float *__restrict__ x32, const float *__restrict__ y32,
                        double *x, double *y)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n + m; i += gridDim.x * blockDim.x) {
        if (i < n) x[i] = (double)x32[i];
        else y[i - n] = (double)y32[i - n];
    }
}

// FP32 copy of FP64 values (round to nearest)
__global__ void k_narrow(int64_t len, const double *__restrict__ src, float *dst)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (float)src[i];
}

// back-map of w_bar (renumbered) to the original LP in its original order:
// x = Pi_C(beta_b D_c xbar), y = beta_c D_r ybar, z = beta_c zbar / D_c
__global__ void k_backmap(int n, int m, double beta_b, double beta_c, const double *xbar,
                          const double *ybar, const double *zbar, const int *perm_c,
                          const int *perm_r, const double *Dr, const double *Dc,
                          const double *lo, const double *uo, double *xo, double *yo, double *zo)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n + m; i += gridDim.x * blockDim.x) {
        if (i < n) {
            const int o = perm_c[i];
            xo[o] = fmin(fmax(beta_b * Dc[o] * xbar[i], lo[o]), uo[o]);
            zo[o] = beta_c * zbar[i] / Dc[o];
        } else {
            const int o = perm_r[i - n];
            yo[o] = beta_c * Dr[o] * ybar[i - n];
        }
    }
}

// dst[i] = src[perm[i]] (into the renumbered order)
__global__ void k_permute(int64_t len, const double *__restrict__ src, const int *__restrict__ perm,
                          double *dst)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[perm[i]];
}

// dst[perm[i]] = src[i] (back to the original order)
__global__ void k_unpermute(int64_t len, const double *__restrict__ src, const int *__restrict__ perm,
                            double *dst)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        dst[perm[i]] = src[i];
}

// stored values of a sliced-ELL matrix from the CSR values (-1: padding, value 0)
__global__ void k_gather_src(int64_t len, const double *__restrict__ csr, int csr_len, const int *__restrict__ src,
                             double *dst)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
        const int p = src[i];
        dst[i] = p >= 0 ? csr[HPR_COL(p, csr_len)] : 0.0;
    }
}

// ------------------------------------------------------------------ power method
// SplitMix64 (Steele, Lea & Flood 2014): i-th output of the stream started at seed
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// u_i = 2 U_{perm[i]} - 1 (the generator is indexed by the original row) and the
// partial ||u||^2 (one partial per CTA)
__global__ void __launch_bounds__(TB) k_pow_start(int m, uint64_t seed, const int *perm, double *u,
                                                  double *partials, int pstride)
{
    __shared__ double red[TB / 32];
    double p = 0.0;
    const int i = blockIdx.x * TB + threadIdx.x;
    if (i < m) {
        const uint64_t o = (uint64_t)(perm ? perm[i] : i);
        const double v = 2.0 * ((double)(splitmix64_at(seed, o) >> 11) * 0x1.0p-53) - 1.0;
        u[i] = v;
        p = v * v;
    }
    const double s = block_sum(p, red);
    if (threadIdx.x == 0) partials[Q_V2 * pstride + blockIdx.x] = s;
}

// after s = A^T u: lambda_k = ||s||^2; stop when |lambda_k - lambda_{k-1}| <= tol lambda_k
__global__ void k_pow_after_s(PowCtl *pc, const double *scal)
{
    if (pc->done) return;
    pc->k += 1;
    pc->lam = scal[Q_S2];
    if (pc->k > 1 && fabs(pc->lam - pc->lam_prev) <= pc->tol * pc->lam) {
        pc->done = 1;
        return;
    }
    pc->lam_prev = pc->lam;
    if (pc->k >= pc->max_iter) pc->stop_after = 1;
}

// after w = A s: 1 / ||w|| for the normalisation
__global__ void k_pow_after_w(PowCtl *pc, const double *scal)
{
    if (pc->done) return;
    const double nw = sqrt(scal[Q_W2]);
    if (!(nw > 0.0)) {
        pc->done = 1;
        return;
    }
    pc->inv = 1.0 / nw;
}

__global__ void k_pow_finish(PowCtl *pc)
{
    if (!pc->done && pc->stop_after) pc->done = 1;
}

// u = w * inv (skipped once done)
__global__ void k_scale_vec(int m, const double *w, double *u, const PowCtl *pc, const double *inv_ptr)
{
    if (pc && pc->done) return;
    const double inv = inv_ptr ? *inv_ptr : pc->inv;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        u[i] = w[i] * inv;
}

__global__ void k_inv_sqrt_scalar(const double *scal, int q, double *out)
{
    *out = 1.0 / sqrt(scal[q]);
}

// ------------------------------------------------------------------ preprocessing
__global__ void k_gather(int64_t nnz, const double *__restrict__ src, const int *__restrict__ perm,
                         double *dst)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
         k += (int64_t)gridDim.x * blockDim.x)
        dst[k] = src[HPR_COL(perm[k], (int)nnz)];
}

// d_i = max_p |val_p| over row i, in index order
__global__ void k_row_absmax(int rows, const int *__restrict__ rp, const double *__restrict__ val,
                             double *d)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += gridDim.x * blockDim.x) {
        double mx = 0.0;
        for (int p = rp[i]; p < rp[i + 1]; ++p) {
            const double a = fabs(val[p]);
            if (a > mx) mx = a;
        }
        d[i] = mx;
    }
}

// d_i = sum_p |val_p|^e over row i, in index order (e == 1: plain |val|)
__global__ void k_row_abspow(int rows, const int *__restrict__ rp, const double *__restrict__ val,
                             double e, double *d)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int p = rp[i]; p < rp[i + 1]; ++p) {
            const double a = fabs(val[p]);
            s += (e == 1.0) ? a : pow(a, e);
        }
        d[i] = s;
    }
}

// d = d > 0 ? 1/sqrt(d) : 1;  D *= d
__global__ void k_factor(int rows, double *d, double *D)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += gridDim.x * blockDim.x) {
        const double v = d[i] > 0.0 ? 1.0 / sqrt(d[i]) : 1.0;
        d[i] = v;
        D[i] *= v;
    }
}

// a_ij <- a_ij * dr_i * dc_j
__global__ void k_scale_rows_cols(int rows, int cols, const int *__restrict__ rp, const int *__restrict__ ci,
                                  double *val, const double *__restrict__ dr,
                                  const double *__restrict__ dc)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += gridDim.x * blockDim.x) {
        const double r = dr[i];
        for (int p = rp[i]; p < rp[i + 1]; ++p) val[p] = val[p] * r * dc[HPR_COL(ci[p], cols)];
    }
}

// b~ = D_r b, c~ = D_c c, l~ = l / D_c, u~ = u / D_c, and the partials of ||b~||^2,
// ||c~||^2 (grid over max(m, n) entries, one partial per CTA)
__global__ void __launch_bounds__(TB) k_prep_vectors(int m, int n, const double *Dr,
                                                     const double *Dc, double *b, double *c,
                                                     double *l, double *u, double *partials,
                                                     int pstride)
{
    __shared__ double red[TB / 32];
    const int i = blockIdx.x * TB + threadIdx.x;
    double pb = 0.0, pcn = 0.0;
    if (i < m) {
        const double v = b[i] * Dr[i];
        b[i] = v;
        pb = v * v;
    }
    if (i < n) {
        const double v = c[i] * Dc[i];
        c[i] = v;
        pcn = v * v;
        l[i] = l[i] / Dc[i];
        u[i] = u[i] / Dc[i];
    }
    double s = block_sum(pb, red);
    if (threadIdx.x == 0) partials[Q_V2 * pstride + blockIdx.x] = s;
    s = block_sum(pcn, red);
    if (threadIdx.x == 0) partials[Q_V2B * pstride + blockIdx.x] = s;
}

// b_s = b~ / beta_b, l_s, u_s likewise, c_s = c~ / beta_c; weights of the residuals in
// the original space w_r = beta_b / D_r, w_c = beta_c / D_c
__global__ void k_prep_normalise(int m, int n, double beta_b, double beta_c, const double *Dr,
                                 const double *Dc, double *b, double *c, double *l, double *u,
                                 double *wr, double *wc)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < (m > n ? m : n);
         i += gridDim.x * blockDim.x) {
        if (i < m) {
            b[i] = b[i] / beta_b;
            wr[i] = beta_b / Dr[i];
        }
        if (i < n) {
            c[i] = c[i] / beta_c;
            l[i] = l[i] / beta_b;
            u[i] = u[i] / beta_b;
            wc[i] = beta_c / Dc[i];
        }
    }
}

__global__ void k_fill(int64_t n, double v, double *d)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        d[i] = v;
}

}  // namespace hprdev
