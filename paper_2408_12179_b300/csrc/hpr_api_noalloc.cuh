// The allocation-free power method (no context, caller-owned buffers).
// Part of the hpr_api.cu translation unit (included once, at its end, so that the kernels
// of hpr_device.cuh are defined once and the file-local helpers are shared).
#pragma once

// ====================================================================== allocation-free power method
//
// For callers that must not allocate device memory (they run under a memory budget
// owned by someone else, or on a pool whose allocator is not theirs).  The call copies a
// control block to the device and synchronises its stream every 16 power steps, so it
// must not be made while its stream is being captured into a CUDA graph.  The LP is theirs, already on the device; this entry point needs only the
// per-CTA partial sums, a few reduced scalars and the power-method control block, and
// keeps them in one fixed array in device global memory that is part of the library
// image.  Every device that loads the library holds that array until the process
// exits; every call on a device shares it.

namespace {

constexpr int NA_SLOTS = 1024;                           // CTAs per reduction, at most
constexpr int NA_PARTIALS = NQ * NA_SLOTS;               // per-CTA partial sums
constexpr int NA_SCAL = NA_PARTIALS;                     // NQ reduced scalars
constexpr int NA_CTL = NA_SCAL + NQ;                     // PowCtl (7 doubles)
constexpr int NA_INV = NA_CTL + 8;                       // 1 / ||u0||
constexpr int NA_DOUBLES = NA_INV + 8;                   // 16,432 doubles = 131,456 bytes

static __device__ __align__(256) double g_noalloc_scratch[NA_DOUBLES];

// Warp-per-row variant of k_spmv_norm: out = M xin, partial ||out||^2 per CTA.  No tile
// schedule is needed, so the caller's plain CSR arrays are enough.
__global__ void __launch_bounds__(TB) k_rows_spmv_norm(int rows, int cols, const int *__restrict__ rp,
                                                       const int *__restrict__ ci,
                                                       const double *__restrict__ val,
                                                       const double *__restrict__ xin, double *out,
                                                       double *partials, int pstride, int q,
                                                       const PowCtl *pc)
{
    __shared__ double red[TB / 32];
    if (pc->done) return;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (TB / 32);
    double p = 0.0;
    // 64-bit counters: rows and row ends may lie within one stride of 2^31
    for (int64_t r = (int64_t)blockIdx.x * (TB / 32) + (threadIdx.x >> 5); r < rows; r += warps) {
        double s = 0.0;
        for (int64_t k = (int64_t)rp[r] + lane; k < (int64_t)rp[r + 1]; k += 32)
            s = fma(val[k], __ldg(xin + HPR_COL(ci[k], cols)), s);
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
    for (int64_t i = (int64_t)blockIdx.x * TB + threadIdx.x; i < m; i += (int64_t)gridDim.x * TB) {
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

// the message stays valid on this thread until its next failing context-free call
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
            k_rows_spmv_norm<<<gT, TB, 0, st>>>((int)n, (int)m, At_row_ptr, At_col_idx, At_val, u, s,
                                                partials, NA_SLOTS, Q_S2, pc);
            k_reduce<<<1, TB, 0, st>>>(partials, NA_SLOTS, rs, scal, &pc->done);
            k_pow_after_s<<<1, 1, 0, st>>>(pc, scal);
            k_rows_spmv_norm<<<gA, TB, 0, st>>>((int)m, (int)n, A_row_ptr, A_col_idx, A_val, s, u,
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
