// Persistent cluster solve: one thread-block cluster of G <= 16 CTAs (one per SM) runs the
// power method and the whole of Algorithm 2 -- iterations, checks every check_every
// iterations, the restart criteria of Section 3.1, SigmaUpdate (Algorithm 3) and the
// termination test of Section 4.1 -- in one launch, for LPs whose data fit in the
// cluster's shared memory.
//
// Everything a normal iteration touches is in shared memory, so an iteration makes no
// L2 or HBM access at all:
//   - each CTA keeps a copy of the slices of A and A^T that its warps own (the same
//     sliced-ELL layouts and the same slice-to-warp assignment as the persistent grid
//     path: warp g takes slices g, g + G*NW, ..., g = warp * G + CTA for A and
//     warp * G + (CTA + G/2) mod G for A^T), with their metadata;
//   - each CTA keeps the state of its own rows: x, x0, c, l, u for the rows of A^T, y0 and
//     b (and the inequality flags) for the rows of A;
//   - every CTA keeps a replica of the two vectors that the SpMVs gather: y (gathered by
//     the x step, eq. update-x) and x_hat (gathered by the y step, eq. update-y-2).  The
//     lane that computes an entry stores it into all G replicas with st.async, each store
//     counting its bytes on the receiving CTA's transaction barrier (mbarrier) for that
//     replica; a CTA gathers from a replica once the barrier's phase for the iteration has
//     completed.  No cluster barrier is needed in a normal iteration (the ordering argument
//     is at the main loop).  The power method uses the same replicas for w and s, with
//     plain remote stores and cluster barriers.
// A check iteration also writes x_bar, z_bar, dx, y_bar, dy to global memory; the check's
// residual passes gather those through L2 after a cluster barrier, and a restart reloads
// the replica of y and the own rows' anchors from them.
//
// The row sums (two FMA chains, even and odd steps, then a fixed butterfly), the updates
// and the per-CTA partial sums are those of the persistent grid path with the same number
// of CTAs, so the two paths give bitwise the same results.  Every wait for a replica's fill
// is bounded: past its budget the CTA raises the error word and leaves the loop, and the
// host reports HPR_ERR_DEVICE_TIMEOUT.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hprgrid {

constexpr int CL_MAX = 16;                    // the largest (non-portable) cluster

// a slice as the cluster kernel keeps it in shared memory
struct SlMeta {
    int r0, r1;                               // its rows (renumbered order)
    int ploc;                                 // its first entry in the CTA's copy of the matrix
    int rloc;                                 // its first row in the CTA's own-row arrays
    int steps, lg;                            // entries per lane; log2 of lanes per row
};

// the largest per-CTA share of the two matrices over the cluster's CTAs (sizes the
// dynamic shared memory, which is the same for every CTA)
struct ClusterDims {
    int entT, entA;                           // stored entries of A^T / A
    int rowsT, rowsA;                         // rows
    int nslT, nslA;                           // slices
};

__host__ __device__ inline size_t cluster_smem_bytes(int m, int n, const ClusterDims &d)
{
    return 8ull * (size_t)(m + n)                          // replicas of y and x_hat
           + 8ull * (size_t)(d.entT + d.entA)              // values
           + 8ull * (5ull * (size_t)d.rowsT + 2ull * (size_t)d.rowsA)   // x, x0, c, l, u; y0, b
           + 4ull * (size_t)(d.entT + d.entA)              // column indices
           + sizeof(SlMeta) * (size_t)(d.nslT + d.nslA)   // slice metadata
           + (size_t)d.rowsA;                              // inequality flags
}

// the cluster's hardware barrier: every thread of every CTA of the cluster arrives
// (release) and waits (acquire), so stores before it -- to global memory or to any CTA's
// shared memory -- are seen by loads after it
__device__ __forceinline__ void cluster_barrier()
{
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

// the shared::cluster address of `local` (a location in this CTA's shared memory) in CTA
// `rank` of the cluster
__device__ __forceinline__ uint32_t peer_addr(const void *local, uint32_t rank)
{
    const uint32_t la = (uint32_t)__cvta_generic_to_shared(local);
    uint32_t ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(la), "r"(rank));
    return ra;
}

__device__ __forceinline__ void st_peer(uint32_t addr, double v)
{
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}

// ---- transaction-count barriers (mbarrier) for the replicas' fills
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *mb, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mb)), "r"(count) : "memory");
}

// makes the initialisation of this CTA's mbarriers visible to the cluster
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// this CTA's one arrival for the current phase, expecting `bytes` of stores into it
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *mb, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mb)), "r"(bytes)
                 : "memory");
}

// whether the phase of parity `parity` has completed (the stores counted by it are visible)
__device__ __forceinline__ bool mbar_try_wait(uint64_t *mb, unsigned parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(mb)), "r"(parity)
        : "memory");
    return ok != 0;
}

// an 8-byte store into a CTA of the cluster that counts 8 bytes on that CTA's mbarrier
// (addresses from peer_addr)
__device__ __forceinline__ void st_async(uint32_t addr, double v, uint32_t mbar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f64 [%0], %1, [%2];" ::"r"(addr), "d"(v),
                 "r"(mbar)
                 : "memory");
}

__device__ __forceinline__ int warp_sum_int(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Copies the slices of M that warp gw owns (gw, gw + GW, ...) into this CTA's shared memory,
// warp after warp in warp order, and calls row_init(row, local row) for each of their rows.
// wtab: 3 * NW ints of shared memory.  Returns the warp's first local slice and its count.
template <class Fr>
__device__ __forceinline__ void cl_stage(const hprsmall::SmallMat &M, int gw, int GW, double *val, int *col,
                                         SlMeta *meta, int *wtab, int *s0, int *ns, Fr row_init)
{
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int cnt = 0, ent = 0, rows = 0;
    for (int s = gw + lane * GW; s < M.nslices; s += 32 * GW) {
        ++cnt;
        ent += __ldg(M.sptr + s + 1) - __ldg(M.sptr + s);
        rows += __ldg(M.srow + s + 1) - __ldg(M.srow + s);
    }
    cnt = warp_sum_int(cnt);
    ent = warp_sum_int(ent);
    rows = warp_sum_int(rows);
    if (lane == 0) {
        wtab[w] = cnt;
        wtab[NW + w] = ent;
        wtab[2 * NW + w] = rows;
    }
    __syncthreads();
    int bs = 0, pe = 0, pr = 0;
    for (int v = 0; v < w; ++v) {
        bs += wtab[v];
        pe += wtab[NW + v];
        pr += wtab[2 * NW + v];
    }
    __syncthreads();                          // wtab is reused by the next call
    int i = 0;
    for (int s = gw; s < M.nslices; s += GW, ++i) {
        const int g0 = __ldg(M.sptr + s), ne = __ldg(M.sptr + s + 1) - g0;
        for (int t = lane; t < ne; t += 32) {
            val[pe + t] = __ldg(M.val + g0 + t);
            col[pe + t] = HPR_COL(__ldg(M.col + g0 + t), M.cols);
        }
        const int r0 = __ldg(M.srow + s), r1 = __ldg(M.srow + s + 1);
        if (lane == 0) meta[bs + i] = SlMeta{r0, r1, pe, pr, ne >> 5, (int)__ldg(M.slg + s)};
        for (int t = lane; t < r1 - r0; t += 32) row_init(r0 + t, pr + t);
        pe += ne;
        pr += r1 - r0;
    }
    *s0 = bs;
    *ns = cnt;
}

// Row sums over this warp's slices (local slices s0 .. s0 + ns - 1) against the vector that
// gx reads: f(row, local row, sum) on the lane that owns the row.  The arithmetic is
// grid_rows's: two FMA chains (even / odd steps), then the fixed xor butterfly.
template <class Gx, class F>
__device__ __forceinline__ void cl_rows(const SlMeta *meta, const double *val, const int *col, int s0, int ns,
                                        Gx gx, F f)
{
    const int lane = threadIdx.x & 31;
    for (int i = 0; i < ns; ++i) {
        const SlMeta sm = meta[s0 + i];
        const int p0 = sm.ploc + lane;
        double a0 = 0.0, a1 = 0.0;
        int k = 0;
        for (; k + 1 < sm.steps; k += 2) {
            const int pa = p0 + (k << 5), pb = pa + 32;
            a0 = fma(val[pa], gx(col[pa]), a0);
            a1 = fma(val[pb], gx(col[pb]), a1);
        }
        if (k < sm.steps) {
            const int pa = p0 + (k << 5);
            a0 = fma(val[pa], gx(col[pa]), a0);
        }
        double sum = sm.steps > 1 ? a0 + a1 : a0;
        for (int o = 1; o < (1 << sm.lg); o <<= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        const int row = sm.r0 + (lane >> sm.lg);
        if ((lane & ((1 << sm.lg) - 1)) == 0 && row < sm.r1) f(row, sm.rloc + (lane >> sm.lg), sum);
    }
}

// g(row, local row) over the rows of this warp's slices
template <class Fg>
__device__ __forceinline__ void cl_own_rows(const SlMeta *meta, int s0, int ns, Fg g)
{
    const int lane = threadIdx.x & 31;
    for (int i = 0; i < ns; ++i) {
        const SlMeta sm = meta[s0 + i];
        for (int t = lane; t < sm.r1 - sm.r0; t += 32) g(sm.r0 + t, sm.rloc + t);
    }
}

// The whole solve of one LP by the CTA of rank `rank` in a cluster of P.G CTAs.
__device__ __forceinline__ void cluster_solve(const GridArgs &P, const ClusterDims &CD, const int rank)
{
    using hprsmall::now_ns;
    const int tid = threadIdx.x, G = P.G;
    // the grid path's warp numbering (A^T's slices start half the cluster further on)
    const int GW = G * NW;
    const int gwA = (tid >> 5) * G + rank, gwT = (tid >> 5) * G + (rank + G / 2) % G;
    const int n = P.n, m = P.m;
    double *xb = P.xb, *zb = P.zb, *dx = P.dx, *yb = P.yb, *dy = P.dy;
    __shared__ double red[NQG * NW];
    __shared__ int s_flag;
    __shared__ double sc[4];                  // power method: 1/||w||, lambda_k
    __shared__ double bc_sigma, bc_ha, bc_hb, bc_ils;
    __shared__ int bc_restart, bc_stop;
    __shared__ double sc_in[2];
    __shared__ uint32_t s_peer_y[CL_MAX], s_peer_xh[CL_MAX];
    __shared__ uint32_t s_peer_mby[CL_MAX], s_peer_mbxh[CL_MAX];
    __shared__ __align__(8) uint64_t mb_y, mb_xh;   // fills of the replicas (one phase each per iteration)
    __shared__ int s_err;
    __shared__ int wtab[3 * NW];
    extern __shared__ __align__(16) unsigned char cl_smem[];
    double *const s_y = reinterpret_cast<double *>(cl_smem);    // replica of y (m)
    double *const s_xh = s_y + m;                                // replica of x_hat (n)
    double *const valT = s_xh + n, *const valA = valT + CD.entT;
    double *const ox = valA + CD.entA, *const ox0 = ox + CD.rowsT, *const oc = ox0 + CD.rowsT;
    double *const ol = oc + CD.rowsT, *const ou = ol + CD.rowsT;
    double *const oy0 = ou + CD.rowsT, *const ob = oy0 + CD.rowsA;
    int *const colT = reinterpret_cast<int *>(ob + CD.rowsA), *const colA = colT + CD.entT;
    SlMeta *const metaT = reinterpret_cast<SlMeta *>(colA + CD.entA), *const metaA = metaT + CD.nslT;
    unsigned char *const oineq = reinterpret_cast<unsigned char *>(metaA + CD.nslA);
    const uint64_t t_start = now_ns();

    int sT0, nT, sA0, nA;
    cl_stage(P.T, gwT, GW, valT, colT, metaT, wtab, &sT0, &nT, [&](int j, int lj) {
        ox[lj] = 0.0;                         // Algorithm 2 from the origin (Section 4.1)
        ox0[lj] = 0.0;
        oc[lj] = __ldg(P.c + j);
        ol[lj] = __ldg(P.l + j);
        ou[lj] = __ldg(P.u + j);
    });
    cl_stage(P.A, gwA, GW, valA, colA, metaA, wtab, &sA0, &nA, [&](int i, int li) {
        oy0[li] = 0.0;
        ob[li] = __ldg(P.b + i);
        oineq[li] = __ldg(P.ineq + i);
    });
    if (tid == 0) {
        mbar_init(&mb_y, 1);
        mbar_init(&mb_xh, 1);
        fence_mbar_init();
        s_err = 0;
    }
    if (tid < G) {
        s_peer_y[tid] = peer_addr(s_y, tid);
        s_peer_xh[tid] = peer_addr(s_xh, tid);
        s_peer_mby[tid] = peer_addr(&mb_y, tid);
        s_peer_mbxh[tid] = peer_addr(&mb_xh, tid);
    }
    cluster_barrier();                        // every CTA runs, and its mbarriers are set, before
                                              // any store to a peer

    // entry idx of a replica, in every CTA of the cluster (this one included)
    auto bcast = [&](const uint32_t *peer, int idx, double v) {
        for (int d = 0; d < G; ++d) st_peer(peer[d] + 8u * (uint32_t)idx, v);
    };
    auto rowsT = [&](auto gx, auto f) { cl_rows(metaT, valT, colT, sT0, nT, gx, f); };
    auto rowsA = [&](auto gx, auto f) { cl_rows(metaA, valA, colA, sA0, nA, gx, f); };
    auto from_y = [&](int c) { return s_y[c]; };
    auto from_xh = [&](int c) { return s_xh[c]; };

    // ---- lambda of T1 = lambda I - A A^* (power method of Section 4.1, counted in the solve
    // time): w in the replica of y, s = A^T w / ||w|| in the replica of x_hat
    double lambda = P.lambda_fixed;
    int64_t piters = 0;
    double prel = 0.0;
    if (!(lambda > 0.0)) {
        double p[1] = {0.0};
        for (int i = rank * NT + tid; i < m; i += G * NT) {
            const double v = 2.0 * ((double)(hprdev::splitmix64_at(P.seed, (uint64_t)P.perm_r[i]) >> 11) * 0x1.0p-53) - 1.0;
            bcast(s_peer_y, i, v);
            p[0] = fma(v, v, p[0]);
        }
        cta_publish<1>(p, red, P.partials, G, rank);
        cluster_barrier();
        grid_sums_then<1>(P.partials, G, [&](const double *sum) {
            sc[0] = 1.0 / sqrt(sum[0]);
            sc[1] = 0.0;
            s_flag = 0;
        });
        __syncthreads();
        int64_t k = 0;
        for (;;) {
            const double inv = sc[0];
            double q[2] = {0.0, 0.0};
            rowsT(from_y, [&](int j, int, double sj) {
                const double t = sj * inv;
                bcast(s_peer_xh, j, t);
                q[0] = fma(t, t, q[0]);
            });
            cluster_barrier();
            rowsA(from_xh, [&](int i, int, double wi) {
                bcast(s_peer_y, i, wi);
                q[1] = fma(wi, wi, q[1]);
            });
            ++k;
            cta_publish<2>(q, red, P.partials, G, rank);
            cluster_barrier();
            grid_sums_then<2>(P.partials, G, [&](const double *sum) {
                const double l = sum[0], prev = sc[1];
                sc[1] = l;
                if (k > 1) sc[2] = fabs(l - prev) / l;
                if ((k > 1 && fabs(l - prev) <= P.power_tol * l) || k >= P.power_max_iter || !(sum[1] > 0.0))
                    s_flag = 1;
                else
                    sc[0] = 1.0 / sqrt(sum[1]);
            });
            __syncthreads();
            if (s_flag) break;
        }
        lambda = sc[1];
        piters = k;
        prel = k > 1 ? sc[2] : 0.0;
    }
    const uint64_t t_power = now_ns();

    auto set_weights = [&](int64_t tn_) {
        volatile double *v = sc_in;
        v[0] = (double)tn_ + 2.0;
        const double d0 = v[0];
        bc_ha = P.halpern ? 1.0 / d0 : 0.0;
        bc_hb = P.halpern ? (d0 - 1.0) / d0 : 1.0;
    };
    auto set_sigma = [&](double sg) {
        volatile double *v = sc_in;
        bc_sigma = sg;
        v[1] = lambda * sg;
        bc_ils = 1.0 / v[1];
    };
    if (tid == 0) {
        set_sigma(P.sigma0);
        set_weights(0);
    }
    // y = 0 in this CTA's replica (the peers' last power-method stores into it came before
    // the last barrier; none comes before the y step of the first iteration)
    for (int i = tid; i < m; i += NT) s_y[i] = 0.0;
    cluster_barrier();

    // Normal iterations run without cluster barriers: each replica's fill for an iteration
    // is one phase of its mbarrier (this CTA's one arrival expecting 8 bytes per entry, and
    // every entry stored into it by st.async, which counts its bytes there); a CTA waits for
    // the phase before it gathers.  No replica is refilled while a CTA still gathers from it:
    // a CTA sends x_hat(k+1) only once its replica of y(k) is complete, that is after every
    // warp of every CTA has sent its rows of y(k), each after its own gathers of x_hat(k); and
    // the same for y.  Each wait is bounded (P.budget_ns): past it the CTA raises the error
    // word and leaves the loop, and every CTA still meets the others at the final barrier.
    unsigned par_y = 0, par_xh = 0;           // parity of each mbarrier's current phase
    bool y_pending = false;                   // a fill of the replica of y is under way
    auto fill_done = [&](uint64_t *mb, unsigned bytes, unsigned &par, int64_t where) -> bool {
        if (tid == 0) mbar_arrive_expect_tx(mb, bytes);
        const uint64_t t0 = now_ns();
        unsigned polls = 0;
        while (!mbar_try_wait(mb, par)) {
            if ((++polls & 63u) == 0 && now_ns() - t0 > P.budget_ns) {
                if (atomicExch(&P.bar->err, 1) == 0) P.bar->where = (int)where;
                s_err = 1;
                break;
            }
        }
        par ^= 1u;
        __syncthreads();
        return s_err == 0;
    };
    auto bcast_async = [&](const uint32_t *peer, const uint32_t *peer_mb, int idx, double v) {
        for (int d = 0; d < G; ++d) st_async(peer[d] + 8u * (uint32_t)idx, v, peer_mb[d]);
    };

    int64_t k = 0;
    OuterState D;
    int64_t t_all = 0;
    int64_t to_check = P.check_every;
#pragma unroll 1
    for (k = 0; k < P.max_iter; ++k) {
        if (y_pending) {                      // y(k) complete in this CTA's replica
            if (!fill_done(&mb_y, 8u * (unsigned)m, par_y, k)) break;
            y_pending = false;
        }
        const double sigma = bc_sigma, ha = bc_ha, hb = bc_hb, inv_ls = bc_ils;
        const bool periodic = (--to_check == 0);
        if (periodic) to_check = P.check_every;
        const bool is_check = periodic || (k + 1 == P.max_iter);
        const bool is_r0 = (t_all == 0);
        const bool store = is_check || is_r0;
        double q[NQG] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        // x step: eq. (update-x), reflection, Halpern step
        rowsT(from_y, [&](int j, int lj, double sj) {
            const double xj = ox[lj], x0j = ox0[lj];
            const double cj = oc[lj], lj_ = ol[lj], uj = ou[lj];
            const double v = fma(sigma, sj - cj, xj);
            const double xbj = hprdev::clamp_lu(v, lj_, uj);
            const double xhj = fma(2.0, xbj, -xj);
            if (!(rank == P.skip_cta && k == (int64_t)P.skip_at))      // fault injection: a lost fill
                bcast_async(s_peer_xh, s_peer_mbxh, j, xhj);
            ox[lj] = fma(hb, P.reflect ? xhj : xbj, ha * x0j);
            if (store) {
                const double zbj = (xbj - v) / sigma, d = xj - xbj, e = xbj - x0j;
                __stcg(xb + j, xbj);
                __stcg(zb + j, zbj);
                __stcg(dx + j, d);
                q[0] = fma(d, d, q[0]);
                q[1] = fma(e, e, q[1]);
                q[2] = fma(cj, xbj, q[2]);
                if (zbj > 0.0) q[3] = fma(zbj, lj_, q[3]);
                else if (zbj < 0.0) q[3] = fma(zbj, uj, q[3]);
            }
        });
        if (!fill_done(&mb_xh, 8u * (unsigned)n, par_xh, k)) break;   // x_hat(k) complete
        // the next iteration's weights, by the last thread while the others update y: every
        // thread of this CTA read this iteration's values before the wait above
        if (!store && tid == NT - 1) set_weights(t_all + 1);
        // y step: eq. (update-y-2), projection on D, reflection, Halpern step
        rowsA(from_xh, [&](int i, int li, double qi) {
            const double yi = s_y[i], y0i = oy0[li];
            const double bi = ob[li];
            double ybi = fma(bi - qi, inv_ls, yi);
            if (oineq[li]) ybi = hprdev::pos_part(ybi);
            const double yhi = fma(2.0, ybi, -yi);
            bcast_async(s_peer_y, s_peer_mby, i, fma(hb, P.reflect ? yhi : ybi, ha * y0i));
            if (store) {
                const double d = yi - ybi, e = ybi - y0i;
                __stcg(yb + i, ybi);
                __stcg(dy + i, d);
                q[4] = fma(d, d, q[4]);
                q[5] = fma(e, e, q[5]);
                q[6] = fma(bi, ybi, q[6]);
            }
        });
        y_pending = true;
        if (!store) {
            ++t_all;
            continue;
        }
        cluster_barrier();                    // the check's global stores, seen by every CTA
        // the check quantities: residual passes in the original-space weights, <dy, A dx>
        rowsT([&](int c) { return __ldcg(yb + c); }, [&](int j, int lj, double sj) {
            const double rj = __ldg(P.wc + j) * (oc[lj] - sj - __ldcg(zb + j));
            q[7] = fma(rj, rj, q[7]);
        });
        rowsA([&](int c) { return __ldcg(xb + c); }, [&](int i, int li, double si) {
            double ri = ob[li] - si;
            if (oineq[li]) ri = hprdev::pos_part(ri);
            ri *= __ldg(P.wr + i);
            q[8] = fma(ri, ri, q[8]);
        });
        rowsA([&](int c) { return __ldcg(dx + c); }, [&](int i, int, double si) { q[9] = fma(__ldcg(dy + i), si, q[9]); });
        cta_publish<NQG>(q, red, P.partials, G, rank);
        cluster_barrier();
        grid_sums_then<NQG>(P.partials, G, [&](const double *sums) {
            int rs, stp;
            double sn;
            check_decide(P, D, sums, rank, k, t_all, is_r0, is_check, sigma, lambda,
                         1e-9 * (double)(now_ns() - t_start), &rs, &stp, &sn);
            bc_restart = rs;
            bc_stop = stp;
            if (rs) set_sigma(sn);
            set_weights(rs ? 0 : t_all + 1);
        });
        __syncthreads();
        if (bc_stop) {
            ++k;
            break;
        }
        if (bc_restart) {
            // w^{r+1,0} = w_bar (Algorithm 2): the replica of y and the own rows' x, x0, y0
            // take y_bar and x_bar (written before the last two barriers).  The replica's
            // fill with y(k+1) completes first; no peer stores into it again before this CTA
            // has sent its rows of x_hat(k+1).
            t_all = 0;
            if (!fill_done(&mb_y, 8u * (unsigned)m, par_y, k)) break;
            y_pending = false;
            for (int i = tid; i < m; i += NT) s_y[i] = __ldcg(yb + i);
            cl_own_rows(metaT, sT0, nT, [&](int j, int lj) {
                const double v = __ldcg(xb + j);
                ox[lj] = v;
                ox0[lj] = v;
            });
            cl_own_rows(metaA, sA0, nA, [&](int i, int li) { oy0[li] = __ldcg(yb + i); });
            __syncthreads();
        } else {
            ++t_all;
        }
    }
    // no CTA leaves while a peer may still store to it: the last fill of y lands, then the
    // cluster meets (after an error the fill may never complete: its wait is bounded too)
    if (y_pending && s_err == 0) (void)fill_done(&mb_y, 8u * (unsigned)m, par_y, k);
    cluster_barrier();
    if (rank == 0 && tid == 0) write_out(P, D, k, lambda, piters, bc_sigma, prel, t_start, t_power);
}

// one LP: the launch is one cluster (grid = cluster = P.G CTAs)
__global__ void __launch_bounds__(NT, 1) k_solve_cluster(GridArgs P, ClusterDims CD)
{
    cluster_solve(P, CD, (int)blockIdx.x);
}

// a batch: cluster c of the launch solves jobs[c] (every job's P.G is the launch's cluster
// size; the dynamic shared memory is the largest job's)
struct ClusterJob {
    GridArgs P;
    ClusterDims CD;
};

__global__ void __launch_bounds__(NT, 1) k_solve_cluster_batch(const ClusterJob *__restrict__ jobs)
{
    __shared__ ClusterJob job;
    unsigned rank, cid;
    asm("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
    asm("mov.u32 %0, %%clusterid.x;" : "=r"(cid));
    if (threadIdx.x == 0) job = jobs[cid];
    __syncthreads();
    cluster_solve(job.P, job.CD, (int)rank);
}

}  // namespace hprgrid
