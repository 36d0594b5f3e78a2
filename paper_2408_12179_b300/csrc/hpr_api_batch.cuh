// The batched solve: many contexts in lock step (fused launches over one work list, or one
// single-CTA launch with a block per LP).
// Part of the hpr_api.cu translation unit (included once, at its end, so that the kernels
// of hpr_device.cuh are defined once and the file-local helpers are shared).
#pragma once

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
// with one CTA per LP (at most two per SM, the LPs independent of one another), then
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
        c->grid_ctas_used = 0;
        c->path_used = 2;
        const int st = small_collect(c);
        if (st < 0) return st;
        if (st != HPR_OK && status == HPR_OK) status = st;
    }
    b->periods = 0;
    b->fused_launches = 1;
    b->solve_time = now_s() - t0;
    return status;
}

// ---- A batch whose LPs all take the persistent cluster path on their own: grouped by that
// solve's cluster size, one launch per group on a stream of its own, one cluster per LP,
// costliest first (the work estimate of the path choice), so that each result equals the
// LP's own solve bit for bit.  The clusters run at their LP's own pace, which wins while
// they are resident together and loses once they queue for SMs: the batch takes cluster
// launches only when they need at most BATCH_CLUSTER_MAX_WAVES waves of resident clusters
// (cudaOccupancyMaxActiveClusters per launch), else the fused path.  Measured on the batched
// family with m in [500, 1000] (200,000-iteration cap): 16 LPs (about one wave) 0.82 s as
// cluster launches against 2.97 s fused; 64 LPs (about 4 waves) 9.35 s against 4.78 s;
// 128 LPs 12.4 s against 7.3 s; 512 LPs 41.7 s against 20.5 s.  A batch with any
// LP that takes another path runs entirely on the fused path (at 1/10 scale, 352 of 512 LPs
// in cluster launches beside the fused path took 68.9 s against 43.0 s fused: the clusters'
// SMs stay busy with latency-bound iterations while the fused launches stream every LP's
// bytes at bandwidth).
constexpr int BATCH_CLUSTER_MAX_WAVES = 2;
struct BatchClusters {
    std::vector<int> size;                    // per context: its cluster size
    std::vector<cudaStream_t> streams;
    std::vector<hprgrid::ClusterJob *> jobs;  // device job tables, one per launch
    int launches = 0;
    ~BatchClusters()
    {
        for (cudaStream_t st : streams) {
            cudaStreamSynchronize(st);
            cudaStreamDestroy(st);
        }
        for (hprgrid::ClusterJob *j : jobs) cudaFree(j);
    }
};

// the cluster size of the LP's own solve if that solve takes the persistent cluster path
// (hpr_solve's choice), else 0; *d its CTAs' shares
int batch_cluster_size(hpr_ctx *c, size_t limit, hprgrid::ClusterDims *d)
{
    const int64_t p = c->opt.persistent;
    if (p != 1 && p != 4) return 0;
    if (cluster_unfit(c, p == 4)) return 0;
    if (p == 1 && !small_unfit(c, false) && small_fp64_per_iter(c) <= SMALL_FP64_VS_CLUSTER) return 0;
    const int G = cluster_ctas(c);
    if (cluster_dims(c, G, d) != HPR_OK || hprgrid::cluster_smem_bytes((int)c->m, (int)c->n, *d) > limit) return 0;
    return G;
}

// prepares and launches every cluster group (asynchronously) when every LP takes the
// cluster path; bc.launches = 0 otherwise
int batch_cluster_launch(hpr_batch *b, double tol, BatchClusters &bc)
{
    using namespace hprgrid;
    std::vector<hpr_ctx *> &cs = b->ctxs;
    bc.size.assign(cs.size(), 0);
    if (cs.empty()) return HPR_OK;
    const size_t limit = cluster_smem_limit(cs[0]);
    std::map<int, std::vector<std::pair<double, size_t>>> groups;   // size -> (cost, context)
    std::vector<ClusterDims> dims(cs.size());
    for (size_t i = 0; i < cs.size(); ++i) {
        const int G = batch_cluster_size(cs[i], limit, &dims[i]);
        if (G == 0) {                          // not every LP: the whole batch is fused
            bc.size.assign(cs.size(), 0);
            return HPR_OK;
        }
        bc.size[i] = G;
        const double cost = small_fp64_per_iter(cs[i]) + CLUSTER_ROW_WEIGHT * (double)(cs[i]->m + cs[i]->n);
        groups[G].push_back({cost, i});
    }
    if (cudaFuncSetAttribute(k_solve_cluster_batch, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
        cudaFuncSetAttribute(k_solve_cluster_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)limit) != cudaSuccess) {
        g_static_err = "hpr_batch_solve: cluster kernel attributes could not be set";
        return HPR_ERR_CUDA;
    }
    // the waves of resident clusters the launches need (a cluster of a launch that can keep nc
    // clusters resident takes 1/nc of the GPU; the launches run side by side)
    double waves = 0.0;
    for (auto &kv : groups) {
        const int G = kv.first;
        size_t smem = 0;
        for (auto &e : kv.second)
            smem = std::max(smem, cluster_smem_bytes((int)cs[e.second]->m, (int)cs[e.second]->n, dims[e.second]));
        cudaLaunchConfig_t cfg{};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)G;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)(G * kv.second.size()));
        cfg.blockDim = dim3(NT);
        cfg.dynamicSmemBytes = smem;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nc = 0;
        if (cudaOccupancyMaxActiveClusters(&nc, k_solve_cluster_batch, &cfg) != cudaSuccess || nc < 1) {
            (void)cudaGetLastError();
            bc.size.assign(cs.size(), 0);      // not resident: the fused path
            return HPR_OK;
        }
        waves += (double)kv.second.size() / (double)nc;
    }
    if (waves > (double)BATCH_CLUSTER_MAX_WAVES) {
        bc.size.assign(cs.size(), 0);
        return HPR_OK;
    }
    for (auto &kv : groups) {
        const int G = kv.first;
        auto &list = kv.second;
        std::stable_sort(list.begin(), list.end(), [](const auto &a, const auto &b2) { return a.first > b2.first; });
        std::vector<ClusterJob> jobs;
        size_t smem = 0;
        for (auto &e : list) {
            hpr_ctx *c = cs[e.second];
            hprsmall::SmallArgs A;
            size_t smem_small = 0;
            int st = small_prepare(c, tol, A, &smem_small);   // solve state, record and result buffers
            if (st) return st;
            if (!c->grid_partials && (st = dalloc(c, &c->grid_partials, grid_partials_len(c)))) return st;
            if (!c->grid_bar && (st = dalloc(c, &c->grid_bar, 1))) return st;
            if (cudaMemsetAsync(c->grid_bar, 0, sizeof(GridBar), b->stream) != cudaSuccess) {
                g_static_err = "hpr_batch_solve: error word could not be cleared";
                return HPR_ERR_CUDA;
            }
            ClusterJob J{};
            J.P = grid_args(c, A, G);
            J.CD = dims[e.second];
            jobs.push_back(J);
            smem = std::max(smem, cluster_smem_bytes((int)c->m, (int)c->n, J.CD));
        }
        cudaLaunchConfig_t cfg{};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)G;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)(G * jobs.size()));
        cfg.blockDim = dim3(NT);
        cfg.dynamicSmemBytes = smem;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nc = 0;
        if (cudaOccupancyMaxActiveClusters(&nc, k_solve_cluster_batch, &cfg) != cudaSuccess || nc < 1) {
            (void)cudaGetLastError();
            g_static_err = "hpr_batch_solve: no cluster of the batch kernel can be resident";
            return HPR_ERR_CUDA;
        }
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            g_static_err = "hpr_batch_solve: stream creation failed";
            return HPR_ERR_CUDA;
        }
        bc.streams.push_back(st);
        ClusterJob *dj = nullptr;
        if (cudaMalloc((void **)&dj, sizeof(ClusterJob) * jobs.size()) != cudaSuccess) {
            g_static_err = "hpr_batch_solve: cluster job table could not be allocated";
            return HPR_ERR_NOMEM;
        }
        bc.jobs.push_back(dj);
        // the contexts' set-up (small_prepare) ran on the batch's stream: the launch follows it
        if (cudaStreamSynchronize(b->stream) != cudaSuccess ||
            cudaMemcpyAsync(dj, jobs.data(), sizeof(ClusterJob) * jobs.size(), cudaMemcpyHostToDevice, st) != cudaSuccess) {
            g_static_err = "hpr_batch_solve: cluster job table could not be copied";
            return HPR_ERR_CUDA;
        }
        cfg.stream = st;
        if (cudaLaunchKernelEx(&cfg, k_solve_cluster_batch, (const ClusterJob *)dj) != cudaSuccess) {
            g_static_err = "hpr_batch_solve: cluster launch failed";
            return HPR_ERR_CUDA;
        }
        bc.launches += 1;
    }
    return HPR_OK;
}

// waits for the cluster launches and reads their contexts back as after their own solves;
// returns the worst status among them (or an error)
int batch_cluster_collect(hpr_batch *b, BatchClusters &bc, int *worst)
{
    for (cudaStream_t st : bc.streams)
        if (cudaStreamSynchronize(st) != cudaSuccess) {
            g_static_err = "hpr_batch_solve: cluster launch failed";
            return HPR_ERR_CUDA;
        }
    for (size_t i = 0; i < b->ctxs.size(); ++i) {
        if (!bc.size[i]) continue;
        hpr_ctx *c = b->ctxs[i];
        c->grid_ctas_used = bc.size[i];
        c->path_used = 4;
        hprgrid::GridBar hb{};
        if (cudaMemcpy(&hb, c->grid_bar, sizeof hb, cudaMemcpyDeviceToHost) != cudaSuccess) {
            g_static_err = "hpr_batch_solve: error word could not be read";
            return HPR_ERR_CUDA;
        }
        if (hb.err) return cluster_timeout(c, hb);
        const int st = small_collect(c);
        if (st < 0) return st;
        if (st != HPR_OK && *worst == HPR_OK) *worst = st;
    }
    return HPR_OK;
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
    {
        BatchClusters bc;
        const int st0 = batch_cluster_launch(b, tol, bc);
        if (st0) return st0;
        if (bc.launches > 0) {                 // every LP in a cluster launch
            b->fused_launches = bc.launches;
            int worst = HPR_OK;
            const int st1 = batch_cluster_collect(b, bc, &worst);
            b->solve_time = now_s() - t0;
            return st1 ? st1 : worst;
        }
    }
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
        c->grid_ctas_used = 0;
        c->path_used = 0;
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
