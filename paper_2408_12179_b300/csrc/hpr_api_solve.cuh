// The solve: periods of Algorithm 2 on the multi-CTA path (CUDA graphs, host decisions
// once per check period), the persistent single-CTA path, and the C ABI calls that solve
// a context and read its results.
// Part of the hpr_api.cu translation unit (included once, at its end, so that the kernels
// of hpr_device.cuh are defined once and the file-local helpers are shared).
#pragma once

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
    // the gather-tiled x phase's work counters start at zero (k_tile_epi resets them after
    // each k_tile_part; a launch that failed in between would leave them set)
    if (ctx->TX.nblk) CK(cudaMemsetAsync(ctx->TX.ctr, 0, sizeof(unsigned) * (size_t)ctx->TX.nblk, s));

    CK(cudaStreamSynchronize(s));
    SolveState &S = ctx->ss;
    S = SolveState{};
    S.tol = tol;
    S.t0 = now_s();
    ctx->launches = 0;

    // ---- T1 = lambda I - A A^*: power method (counted in the solve time, Section 4.1);
    // a resumed solve takes the checkpoint's lambda
    const bool resume = ctx->resume_pending;
    if (resume) {
        ctx->lambda = ctx->resume_hdr.lambda;
        ctx->power_iters = ctx->resume_hdr.power_iters;
        ctx->power_time = 0.0;
        ctx->power_rel_change = ctx->resume_hdr.power_rel_change;
    } else if (o.lambda_fixed > 0.0) {
        ctx->lambda = o.lambda_fixed;
        ctx->power_iters = 0;
        ctx->power_time = 0.0;
        ctx->power_rel_change = 0.0;
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
    CK(cudaMemsetAsync(ctx->x032, 0, sizeof(float) * n, s));
    CK(cudaMemsetAsync(ctx->y032, 0, sizeof(float) * m, s));
    ctx->form = (int)o.precision;
    S.sigma = o.sigma0;
    S.status = HPR_MAX_ITER;
    if (resume) {
        // the checkpoint: Algorithm 2's restart step applied to its anchor, its sigma and
        // counters (t = 0: a new inner loop)
        const StateHdr &H = ctx->resume_hdr;
        CK(cudaMemcpyAsync(ctx->xbar, ctx->resume_x0.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(ctx->ybar, ctx->resume_y0.data(), sizeof(double) * m, cudaMemcpyHostToDevice, s));
        ctx->form = (int)H.form;
        if (ctx->form == 1)
            k_restart32<<<grid_for(n + m), 256, 0, s>>>((int)n, (int)m, ctx->xbar, ctx->ybar, ctx->x32, ctx->x0,
                                                        ctx->y32, ctx->y0, ctx->x032, ctx->y032);
        else
            k_restart<<<grid_for(n + m), 256, 0, s>>>((int)n, (int)m, ctx->xbar, ctx->ybar, ctx->x, ctx->x0,
                                                      ctx->y, ctx->y0);
        CKL();
        ctx->launches += 1;
        CK(cudaStreamSynchronize(s));
        S.k = H.k;
        S.r = H.r;
        S.sigma = H.sigma;
        ctx->resume_pending = false;
    }
    S.k_restart = S.k;
    S.sigma_restart = S.sigma;
    S.form_restart = ctx->form;
    S.tracing = ctx->trace_n > 0;
    S.done = o.max_iter <= S.k;
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

    if (ctx->fault_nan_check > 0 && ++ctx->check_count == ctx->fault_nan_check)
        ctx->scal_h[NQ + Q_RP] = std::nan("");   // HPR_FAULT_NAN_CHECK: a poisoned read-back
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
                                                    ctx->x0, ctx->y32, ctx->y0, ctx->x032, ctx->y032);
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
        S.k_restart = kk + 1;                // the checkpoint: this restart
        S.sigma_restart = S.sigma;
        S.form_restart = ctx->form;
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
    I.power_rel_change = ctx->power_rel_change;
    I.n_checks = (int64_t)ctx->checks.size(); I.launches = ctx->launches; I.status = S.status;
    I.iters_fp32 = S.iters_fp32;
    I.policy_decisions = S.policy_decisions;
    I.policy_fallbacks = S.policy_fallbacks;
    I.path = ctx->path_used;
    I.path_ctas = ctx->grid_ctas_used;
    I.x_tiles = (ctx->path_used == 0 && !ctx->batched && tiles_on(ctx)) ? ctx->TX.nblk : 0;
    ctx->solved = true;
    return S.status;
}

constexpr size_t SMALL_SMEM_MAX = 200 * 1024;
// One SM issues the FP64 work of the whole iteration: about one warp instruction per 32
// stored entries of A and A^T plus ~8 per 32-row slice (row sums' tails and epilogues), at
// ~17 cycles each.  Measured on the tiny planted LP, QAPs (N = 5, 6) and medium planted LPs
// at 1/1000 .. 1/200 scale, an iteration of the single CTA costs ~1.5 us + 8.4 ns per such
// instruction, and the multi-CTA graph path ~5 us (launch-bound) or more; the default takes
// the single CTA up to 600 instructions (~6.5 us) against the multi-CTA path, and up to 200
// (~3.1 us) when the persistent cluster path can run the LP: one CTA of a cluster issues only
// its share of the FP64 work, and the cluster's iterations cost ~3.3 us and up (measured: the
// tiny planted LP, 172 instructions, 2.85 us in one CTA and 3.33 us in a cluster; the medium
// planted LP at 1/1000 scale, 587 instructions, 7.13 us in one CTA and 3.84 us in a cluster of 4).
constexpr double SMALL_FP64_MAX = 600.0;
constexpr double SMALL_FP64_VS_CLUSTER = 200.0;

double small_fp64_per_iter(const hpr_ctx *ctx)
{
    // one SM issues the FP64 work of an iteration (or of a power step, the same SpMVs)
    return (double)(ctx->SA.entries + ctx->ST.entries) / 32.0 + 8.0 * (double)(ctx->SA.nslices + ctx->ST.nslices);
}

// whether the persistent single-CTA path can run this solve (and why not); unless forced,
// also whether it is expected to be the faster path
const char *small_unfit(const hpr_ctx *ctx, bool forced)
{
    const hpr_options &o = ctx->opt;
    if (ctx->resume_pending) return "a pending resume (hpr_set_state)";
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
        M.nslices = D.nslices; M.cols = D.cols; M.entries = D.entries;
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
    ctx->power_rel_change = h[SO_POWER_REL];
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
    ctx->path_used = 2;
    return small_collect(ctx);
}

// ---------------------------------------------------------------- persistent grid path
// Mid-size LPs: one cooperative launch of G CTAs (hpr_grid.cuh).  Its CTA count follows the
// FP64 work of an iteration (the part's FP64 issue rate bounds each SM's share): about
// GRID_FP64_PER_CTA warp instructions per CTA, at most one CTA per SM.  The default path
// choice takes it between the single-CTA path's limit and GRID_FP64_MAX.
constexpr double GRID_FP64_PER_CTA = 100.0;
constexpr double GRID_FP64_MAX = 0.0;
constexpr uint64_t GRID_BUDGET_NS = 5000000000ull;       // 5 s: longest wait at a barrier
constexpr uint64_t GRID_FAULT_BUDGET_NS = 200000ull;     // 200 us when a skip is injected
constexpr int CLUSTER_MAX_CTAS = 16;                     // the largest (non-portable) cluster
// cluster path: CTAs from the FP64 work of an iteration (about CLUSTER_FP64_PER_CTA warp
// instructions per CTA, 2 to 16), and the largest work it takes by default, counted as the
// FP64 warp instructions of an iteration plus CLUSTER_ROW_WEIGHT per row (each row's value
// is stored into every CTA's replica).  Fit to the measured iterations of eight LPs at 16
// CTAs: about 2.4 us + 0.41 ns per FP64 instruction + 0.20 ns per row.  Per iteration against
// the multi-CTA graph path (3,000 iterations; work in brackets): medium planted LPs at
// 1/1000 .. 1/100 scale 3.8 / 4.2 / 4.4 / 6.6 us against 7.0 / 7.1 / 8.1 / 8.2 (1,000 ..
// 10,400), QAP N = 8 4.4 against 7.0 (6,100), N = 9 5.9 against 6.4 (9,700); left to the
// graph path: the medium LP at 1/80 scale 8.1 against 8.8 (13,000), the multicommodity-flow
// LP with 300 nodes 7.5 against 6.6 (11,600), QAP N = 10 8.3 against 7.4 (14,500).
constexpr double CLUSTER_FP64_PER_CTA = 150.0;
constexpr double CLUSTER_ROW_WEIGHT = 0.48;
constexpr double CLUSTER_WORK_MAX = 10500.0;

const char *grid_unfit(const hpr_ctx *ctx, bool forced)
{
    const hpr_options &o = ctx->opt;
    if (ctx->resume_pending) return "a pending resume (hpr_set_state)";
    if (o.precision != 0) return "the FP32 form";
    if (o.trace_iters > 0) return "tracing";
    if (o.time_limit_s > 0.0) return "a time limit";
    if (o.sigma_policy != 0) return "a sigma policy";
    if (!forced && small_fp64_per_iter(ctx) > GRID_FP64_MAX) return "enough work per iteration to fill the GPU from launches";
    return nullptr;
}

// CTA partial sums of the grid and cluster paths (one buffer serves both)
int64_t grid_partials_len(const hpr_ctx *ctx)
{
    return (int64_t)hprgrid::NQG * std::max(CLUSTER_MAX_CTAS, ctx->num_sms);
}

// the launch arguments of a persistent grid or cluster solve over G CTAs (A from small_prepare)
hprgrid::GridArgs grid_args(hpr_ctx *ctx, const hprsmall::SmallArgs &A, int G)
{
    using namespace hprgrid;
    GridArgs P{};
    P.m = A.m; P.n = A.n; P.G = G;
    P.A = A.A; P.T = A.T;
    P.ineq = A.ineq;
    P.b = A.b; P.c = A.c; P.l = A.l; P.u = A.u; P.wr = A.wr; P.wc = A.wc;
    P.beta_b = A.beta_b; P.beta_c = A.beta_c; P.norm_b = A.norm_b; P.norm_c = A.norm_c;
    P.tol = A.tol; P.alpha1 = A.alpha1; P.alpha2 = A.alpha2; P.alpha3 = A.alpha3; P.sigma0 = A.sigma0;
    P.lambda_fixed = A.lambda_fixed; P.power_tol = A.power_tol;
    P.max_iter = A.max_iter; P.check_every = A.check_every; P.power_max_iter = A.power_max_iter;
    P.seed = A.seed;
    P.restart = A.restart; P.sigma_update = A.sigma_update; P.halpern = A.halpern; P.reflect = A.reflect;
    P.perm_r = A.perm_r;
    P.x = ctx->x; P.x0 = ctx->x0; P.xh = ctx->xhat; P.xb = ctx->xbar; P.zb = ctx->zbar; P.dx = ctx->dx;
    P.y = ctx->y; P.y0 = ctx->y0; P.yb = ctx->ybar; P.dy = ctx->dy;
    P.partials = ctx->grid_partials;
    P.bar = ctx->grid_bar;
    P.budget_ns = ctx->fault_barrier > 0 ? GRID_FAULT_BUDGET_NS : GRID_BUDGET_NS;
    P.skip_cta = ctx->fault_barrier > 0 ? G - 1 : -1;
    P.skip_at = ctx->fault_barrier > 0 ? (int)(ctx->fault_barrier - 1) : -1;
    P.recs = A.recs; P.rec_cap = A.rec_cap; P.out = A.out;
    return P;
}

// the largest per-CTA share of the two sliced-ELL matrices for a cluster of G CTAs, from
// host copies of the slice pointers
int cluster_dims(hpr_ctx *ctx, int G, hprgrid::ClusterDims *out)
{
    using namespace hprgrid;
    hprgrid::ClusterDims d{};
    for (int which = 0; which < 2; ++which) {
        const SellDev &M = which ? ctx->SA : ctx->ST;
        std::vector<int> srow((size_t)M.nslices + 1), sptr((size_t)M.nslices + 1);
        CK(cudaMemcpy(srow.data(), M.srow, sizeof(int) * srow.size(), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(sptr.data(), M.sptr, sizeof(int) * sptr.size(), cudaMemcpyDeviceToHost));
        std::vector<int64_t> ent(G, 0), rows(G, 0), nsl(G, 0);
        for (int sl = 0; sl < M.nslices; ++sl) {
            // warp g owns slices g (mod G * NW); g = warp * G + CTA for A, and
            // warp * G + (CTA + G/2) mod G for A^T
            const int r = (sl % (G * NW)) % G;
            const int cta = which ? r : (r - G / 2 + G) % G;
            ent[cta] += sptr[sl + 1] - sptr[sl];
            rows[cta] += srow[sl + 1] - srow[sl];
            nsl[cta] += 1;
        }
        const int e = (int)*std::max_element(ent.begin(), ent.end());
        const int r = (int)*std::max_element(rows.begin(), rows.end());
        const int q = (int)*std::max_element(nsl.begin(), nsl.end());
        if (which) { d.entA = e; d.rowsA = r; d.nslA = q; }
        else { d.entT = e; d.rowsT = r; d.nslT = q; }
    }
    *out = d;
    return HPR_OK;
}

// the cluster size of a solve: from the FP64 work of an iteration, or HPR_GRID_CTAS
int cluster_ctas(const hpr_ctx *ctx)
{
    int G = (int)std::ceil(small_fp64_per_iter(ctx) / CLUSTER_FP64_PER_CTA);
    if (ctx->grid_ctas_env > 0) G = (int)std::min<int64_t>(ctx->grid_ctas_env, CLUSTER_MAX_CTAS);
    return std::max(2, std::min(G, CLUSTER_MAX_CTAS));
}

// the dynamic shared memory one CTA of the cluster kernels may have (the opt-in limit less
// the larger static shared memory of the solo and the batch kernel)
size_t cluster_smem_limit(const hpr_ctx *ctx)
{
    cudaFuncAttributes fa{}, fb{};
    int optin = 0;
    if (cudaFuncGetAttributes(&fa, hprgrid::k_solve_cluster) != cudaSuccess ||
        cudaFuncGetAttributes(&fb, hprgrid::k_solve_cluster_batch) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    const size_t st = std::max(fa.sharedSizeBytes, fb.sharedSizeBytes);
    return (size_t)optin > st ? (size_t)optin - st : 0;
}

// whether the persistent cluster path can run this solve (and why not); unless forced, also
// whether it is expected to be the faster path
const char *cluster_unfit(hpr_ctx *ctx, bool forced)
{
    if (const char *why = grid_unfit(ctx, true)) return why;
    if (!forced && small_fp64_per_iter(ctx) + CLUSTER_ROW_WEIGHT * (double)(ctx->m + ctx->n) > CLUSTER_WORK_MAX)
        return "enough work per iteration to fill the GPU from launches";
    const size_t limit = cluster_smem_limit(ctx);
    const int G = cluster_ctas(ctx);
    // a lower bound first (replicas and an even share of the matrices), then the exact need
    const size_t lower = 8ull * (size_t)(ctx->m + ctx->n) + 12ull * (size_t)(ctx->SA.entries + ctx->ST.entries) / G;
    hprgrid::ClusterDims d{};
    if (lower > limit || cluster_dims(ctx, G, &d) != HPR_OK ||
        hprgrid::cluster_smem_bytes((int)ctx->m, (int)ctx->n, d) > limit)
        return "the LP does not fit in the shared memory of the cluster";
    return nullptr;
}

// a wait of the cluster path for a replica's fill ran out of its time budget
int cluster_timeout(hpr_ctx *ctx, const hprgrid::GridBar &hb)
{
    return fail_arg(ctx, HPR_ERR_DEVICE_TIMEOUT,
                    "persistent cluster solve: a wait for a replica's fill at iteration " + std::to_string(hb.where) +
                        " ran out of its time budget; every CTA left the loop");
}

int solve_cluster(hpr_ctx *ctx, double tol)
{
    using namespace hprgrid;
    hprsmall::SmallArgs A;
    size_t smem_small = 0;
    int st = small_prepare(ctx, tol, A, &smem_small);   // solve state, record and result buffers
    if (st) return st;
    CK(cudaFuncSetAttribute(k_solve_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    const size_t limit = cluster_smem_limit(ctx);
    CK(cudaFuncSetAttribute(k_solve_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)limit));
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    cfg.blockDim = dim3(NT);
    cfg.stream = ctx->stream;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    ClusterDims d{};
    int G = cluster_ctas(ctx);
    for (; G >= 2; --G) {                    // the largest resident cluster up to G that fits
        if ((st = cluster_dims(ctx, G, &d))) return st;
        const size_t smem = cluster_smem_bytes((int)ctx->m, (int)ctx->n, d);
        if (smem > limit) break;             // fewer CTAs only take larger shares
        cfg.gridDim = dim3(G);
        cfg.dynamicSmemBytes = smem;
        at[0].val.clusterDim.x = (unsigned)G;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        int nc = 0;
        if (cudaOccupancyMaxActiveClusters(&nc, k_solve_cluster, &cfg) == cudaSuccess && nc >= 1) break;
        (void)cudaGetLastError();
    }
    if (G < 2 || cfg.dynamicSmemBytes == 0 || cluster_smem_bytes((int)ctx->m, (int)ctx->n, d) > limit)
        return fail_arg(ctx, HPR_ERR_ARG, "persistent cluster path: no cluster of two or more CTAs holds the LP");
    if (!ctx->grid_partials) DALLOC(ctx->grid_partials, grid_partials_len(ctx));
    if (!ctx->grid_bar) DALLOC(ctx->grid_bar, 1);
    GridArgs P = grid_args(ctx, A, G);
    CK(cudaMemsetAsync(ctx->grid_bar, 0, sizeof(GridBar), ctx->stream));
    CK(cudaLaunchKernelEx(&cfg, k_solve_cluster, P, d));
    GridBar hb{};
    CK(cudaMemcpyAsync(&hb, ctx->grid_bar, sizeof hb, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->grid_ctas_used = G;
    ctx->path_used = 4;
    if (hb.err) return cluster_timeout(ctx, hb);
    return small_collect(ctx);
}

int solve_grid(hpr_ctx *ctx, double tol)
{
    using namespace hprgrid;
    hprsmall::SmallArgs A;
    size_t smem = 0;
    int st = small_prepare(ctx, tol, A, &smem);   // solve state, record and result buffers
    if (st) return st;
    int per_sm = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve_grid, NT, 0));
    if (per_sm < 1) return fail_arg(ctx, HPR_ERR_CUDA, "the persistent grid kernel does not fit on an SM");
    const int maxG = std::max(1, ctx->num_sms);
    int G = (int)std::ceil(small_fp64_per_iter(ctx) / GRID_FP64_PER_CTA);
    if (ctx->grid_ctas_env > 0) G = (int)std::min<int64_t>(ctx->grid_ctas_env, maxG);
    G = std::max(2, std::min(G, maxG));
    if (!ctx->grid_partials) DALLOC(ctx->grid_partials, grid_partials_len(ctx));
    if (!ctx->grid_bar) DALLOC(ctx->grid_bar, 1);
    GridArgs P = grid_args(ctx, A, G);
    CK(cudaMemsetAsync(ctx->grid_bar, 0, sizeof(GridBar), ctx->stream));
    void *kargs[] = {&P};
    CK(cudaLaunchCooperativeKernel((const void *)k_solve_grid, dim3(G), dim3(NT), kargs, 0, ctx->stream));
    GridBar hb{};
    CK(cudaMemcpyAsync(&hb, ctx->grid_bar, sizeof hb, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->grid_ctas_used = G;
    ctx->path_used = 3;
    if (hb.err)
        return fail_arg(ctx, HPR_ERR_DEVICE_TIMEOUT,
                        "persistent grid solve: a wait at grid barrier " + std::to_string(hb.where) +
                            " ran out of its time budget; every CTA returned");
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
    ctx->grid_ctas_used = 0;
    ctx->path_used = 0;
    if (ctx->opt.persistent == 1 || ctx->opt.persistent == 2) {
        const char *why = small_unfit(ctx, ctx->opt.persistent == 2);
        if (!why && ctx->opt.persistent == 1 && small_fp64_per_iter(ctx) > SMALL_FP64_VS_CLUSTER &&
            !cluster_unfit(ctx, false))
            why = "the persistent cluster path is faster";
        if (!why) return solve_small(ctx, tol);
        if (ctx->opt.persistent == 2)
            return fail_arg(ctx, HPR_ERR_ARG, std::string("persistent = 2 but the single-CTA path cannot run: ") + why);
    }
    if (ctx->opt.persistent == 1 || ctx->opt.persistent == 4) {
        const char *why = cluster_unfit(ctx, ctx->opt.persistent == 4);
        if (!why) return solve_cluster(ctx, tol);
        if (ctx->opt.persistent == 4)
            return fail_arg(ctx, HPR_ERR_ARG, std::string("persistent = 4 but the persistent cluster path cannot run: ") + why);
    }
    if (ctx->opt.persistent == 1 || ctx->opt.persistent == 3) {
        const char *why = grid_unfit(ctx, ctx->opt.persistent == 3);
        if (!why) return solve_grid(ctx, tol);
        if (ctx->opt.persistent == 3)
            return fail_arg(ctx, HPR_ERR_ARG, std::string("persistent = 3 but the persistent grid path cannot run: ") + why);
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

int hpr_get_state(const hpr_ctx *cctx, void *buf, int64_t bytes, int64_t *needed)
{
    if (!cctx) return HPR_ERR_ARG;
    hpr_ctx *ctx = const_cast<hpr_ctx *>(cctx);
    const int64_t n = ctx->n, m = ctx->m;
    const int64_t need = (int64_t)sizeof(StateHdr) + (int64_t)sizeof(double) * (n + m);
    if (needed) *needed = need;
    if (!buf) return HPR_OK;
    if (!ctx->solved) return fail_arg(ctx, HPR_ERR_STATE, "hpr_get_state: no solve has completed");
    if (ctx->path_used != 0)
        return fail_arg(ctx, HPR_ERR_STATE,
                        "hpr_get_state: the last solve ran on a persistent path (its anchors stay in shared "
                        "memory); solve with persistent = 0 to take a checkpoint");
    if (bytes < need) return fail_arg(ctx, HPR_ERR_ARG, "hpr_get_state: the buffer is smaller than needed");
    cudaSetDevice(ctx->device);
    const SolveState &S = ctx->ss;
    StateHdr H{};
    H.magic = STATE_MAGIC;
    H.n = n; H.m = m; H.m1 = ctx->m1; H.nnz = ctx->nnz;
    H.precision = ctx->opt.precision; H.check_every = ctx->opt.check_every;
    H.beta_b = ctx->beta_b; H.beta_c = ctx->beta_c; H.norm_b = ctx->norm_b; H.norm_c = ctx->norm_c;
    H.k = S.k_restart; H.r = S.r; H.form = S.form_restart; H.power_iters = ctx->power_iters;
    H.sigma = S.sigma_restart; H.lambda = S.lambda; H.power_rel_change = ctx->power_rel_change;
    char *out = static_cast<char *>(buf);
    memcpy(out, &H, sizeof H);
    double *x0 = reinterpret_cast<double *>(out + sizeof H);
    CK(cudaMemcpyAsync(x0, ctx->x0, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(x0 + n, ctx->y0, sizeof(double) * m, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return HPR_OK;
}

int hpr_set_state(hpr_ctx *ctx, const void *buf, int64_t bytes)
{
    if (!ctx) return HPR_ERR_ARG;
    if (!buf) return fail_arg(ctx, HPR_ERR_ARG, "hpr_set_state: buf is NULL");
    if (ctx->batched) return fail_arg(ctx, HPR_ERR_STATE, "hpr_set_state: the context belongs to a batch");
    if (ctx->opt.trace_iters > 0 || ctx->opt.sigma_policy != 0)
        return fail_arg(ctx, HPR_ERR_STATE, "hpr_set_state: tracing and a sigma policy cannot resume");
    const int64_t n = ctx->n, m = ctx->m;
    const int64_t need = (int64_t)sizeof(StateHdr) + (int64_t)sizeof(double) * (n + m);
    if (bytes < (int64_t)sizeof(StateHdr) || bytes < need)
        return fail_arg(ctx, HPR_ERR_ARG, "hpr_set_state: the blob is shorter than this LP's state");
    StateHdr H;
    memcpy(&H, buf, sizeof H);
    if (H.magic != STATE_MAGIC) return fail_arg(ctx, HPR_ERR_ARG, "hpr_set_state: not a state blob of this build");
    if (H.n != n || H.m != m || H.m1 != ctx->m1 || H.nnz != ctx->nnz || H.beta_b != ctx->beta_b ||
        H.beta_c != ctx->beta_c || H.norm_b != ctx->norm_b || H.norm_c != ctx->norm_c)
        return fail_arg(ctx, HPR_ERR_ARG, "hpr_set_state: the state was taken from another LP");
    if (H.precision != ctx->opt.precision || H.check_every != ctx->opt.check_every)
        return fail_arg(ctx, HPR_ERR_ARG, "hpr_set_state: the state was taken with another precision or check_every");
    if (!(H.lambda > 0.0) || !(H.sigma > 0.0) || H.k < 0 || H.r < 0 || H.form < 0 || H.form > 1)
        return fail_arg(ctx, HPR_ERR_ARG, "hpr_set_state: inconsistent state");
    const double *x0 = reinterpret_cast<const double *>(static_cast<const char *>(buf) + sizeof H);
    ctx->resume_x0.assign(x0, x0 + n);
    ctx->resume_y0.assign(x0 + n, x0 + n + m);
    ctx->resume_hdr = H;
    ctx->resume_pending = true;
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

int hpr_tile_plan(const hpr_csr *B, int64_t tile_len, int64_t grid, int64_t *sizes, int32_t *row_order,
                  int32_t *bstart, int32_t *ustart, int32_t *cta_blk, int32_t *wstart, int32_t *smeta,
                  int32_t *oslot, int32_t *slot_ptr, uint16_t *col, int32_t *src)
{
    if (!B || B->rows < 1 || B->cols < 1 || B->nnz < 0 || B->rows >= (int64_t)INT32_MAX ||
        B->cols >= (int64_t)INT32_MAX || B->nnz >= (int64_t)INT32_MAX || !B->row_ptr ||
        (B->nnz > 0 && !B->col_idx) || tile_len < 2 || tile_len > 65536 || grid < 1 || grid > 65536) {
        g_static_err = "hpr_tile_plan: bad matrix or parameters";
        return HPR_ERR_ARG;
    }
    const int rows = (int)B->rows;
    if (B->row_ptr[0] != 0 || B->row_ptr[rows] != B->nnz) {
        g_static_err = "hpr_tile_plan: row_ptr[0] != 0 or row_ptr[rows] != nnz";
        return HPR_ERR_ARG;
    }
    std::vector<int> rp((size_t)rows + 1), ci((size_t)std::max<int64_t>(B->nnz, 1), 0), icol((size_t)B->cols);
    for (int i = 0; i <= rows; ++i) {
        rp[(size_t)i] = (int)B->row_ptr[i];
        if (i > 0 && rp[(size_t)i] < rp[(size_t)i - 1]) {
            g_static_err = "hpr_tile_plan: row_ptr decreases";
            return HPR_ERR_ARG;
        }
    }
    for (int64_t p = 0; p < B->nnz; ++p) {
        if (B->col_idx[p] < 0 || B->col_idx[p] >= B->cols) {
            g_static_err = "hpr_tile_plan: column index out of range";
            return HPR_ERR_ARG;
        }
        ci[(size_t)p] = B->col_idx[p];
    }
    for (int64_t j = 0; j < B->cols; ++j) icol[(size_t)j] = (int)j;
    const std::vector<int> perm = order_by_length(rp, rows);
    TileHost H;
    if (!build_tiles(rp, ci, rows, perm, icol, (int)B->cols, (int)tile_len, (int)grid, SELL_STEPS, UNIT_COST, H)) {
        g_static_err = "hpr_tile_plan: the blocks would outnumber the grid's CTAs (or 256), or the offsets exceed 32 bits";
        return HPR_ERR_ARG;
    }
    if (sizes) {
        sizes[0] = H.nblk;
        sizes[1] = (int64_t)H.smeta.size();
        sizes[2] = (int64_t)H.col.size();
        sizes[3] = (int64_t)H.oslot.size();
        sizes[4] = (int64_t)H.wstart.size() - 1;
        sizes[5] = (int64_t)H.cta_blk.size();
    }
    auto put = [](int32_t *dst, const std::vector<int> &v) {
        if (dst && !v.empty()) memcpy(dst, v.data(), sizeof(int32_t) * v.size());
    };
    put(row_order, perm);
    put(bstart, H.bstart);
    put(ustart, H.ustart);
    put(cta_blk, H.cta_blk);
    put(wstart, H.wstart);
    put(oslot, H.oslot);
    put(slot_ptr, H.slot_ptr);
    put(src, H.src);
    if (smeta && !H.smeta.empty()) memcpy(smeta, H.smeta.data(), sizeof(int4) * H.smeta.size());
    if (col && !H.col.empty()) memcpy(col, H.col.data(), sizeof(uint16_t) * H.col.size());
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
    if (ctx->TX.nblk) CK(cudaMemsetAsync(ctx->TX.ctr, 0, sizeof(unsigned) * (size_t)ctx->TX.nblk, s));
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
    const int form_saved = ctx->form;
    ctx->form = ctx->opt.precision == 1 ? 1 : 0;
    if (rc == HPR_OK) rc = (cudaEventRecord(ev[0], s) == cudaSuccess) ? HPR_OK : HPR_ERR_CUDA;
    for (int64_t r = 0; r < total && rc == HPR_OK; ++r) {
        // the kernels of a normal iteration of a solve (an event between two launches makes
        // the programmatic overlap between them a plain stream order)
        rc = launch_normal_x(ctx, 0);
        if (rc) break;
        cudaEventRecord(ev[(size_t)(2 * r + 1)], s);
        rc = launch_normal_y(ctx, 0);
        if (rc) break;
        cudaEventRecord(ev[(size_t)(2 * r + 2)], s);
    }
    ctx->form = form_saved;
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
