// Memory-system probe for the benchmark's roofline (no counterpart in the paper).
// Part of the hpr_api.cu translation unit (included once, at its end).
//
// Two figures bound the SpMV phases on this part: HBM bandwidth for the streamed arrays, and
// the rate of random 8-byte gathers, each of which costs the L1 a cache-tag lookup whatever
// the number of bytes used.  This probe measures both with kernels whose consumers stay off
// the FP64 pipe (integer XOR), so that neither figure is capped by FP64 issue.
#pragma once

namespace {

__device__ __forceinline__ uint32_t probe_hash(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

// read-only stream: four independent 16-byte loads in flight per thread, XOR-consumed
__global__ void __launch_bounds__(256) k_probe_read(const uint4 *__restrict__ a, int64_t n, unsigned *out)
{
    unsigned acc = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n; i += 4 * stride) {
        uint4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = __ldcs(a + i + u * stride);
#pragma unroll
        for (int u = 0; u < 4; ++u) acc ^= v[u].x ^ v[u].y ^ v[u].z ^ v[u].w;
    }
    for (; i < n; i += stride) {
        const uint4 v = __ldcs(a + i);
        acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
    if (acc == 0x9e3779b9u) out[0] = acc;     // keeps the loads; practically never taken
}

// random 8-byte gathers from x[0 .. len) (len a power of two), indices hashed in registers
__global__ void __launch_bounds__(256) k_probe_gather(const double *__restrict__ x, uint32_t mask, int rounds,
                                                      unsigned long long *out)
{
    unsigned long long acc = 0;
    uint32_t h = probe_hash(blockIdx.x * 256u + threadIdx.x + 1u);
    for (int r = 0; r < rounds; ++r) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            h = probe_hash(h + (uint32_t)u);
            v[u] = __ldg(x + (h & mask));
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) acc ^= (unsigned long long)__double_as_longlong(v[u]);
    }
    if (acc == 0x9e3779b97f4a7c15ull) out[0] = acc;
}

// FP64 issue: eight independent DFMA chains per thread (a dependent DFMA takes ~70 cycles,
// so a few warps per SM keep the FP64 pipe issuing every cycle it can)
__global__ void __launch_bounds__(256) k_probe_fp64(int rounds, double *out)
{
    double a[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u] = 1.0 + 1e-3 * (double)(threadIdx.x + 32 * u);
    const double mul = 0.9999999999, add = 1e-12;
    for (int r = 0; r < rounds; ++r) {
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] = fma(a[u], mul, add);
    }
    double s = a[0];
#pragma unroll
    for (int u = 1; u < 8; ++u) s += a[u];
    if (s == 1234.5678) out[0] = s;          // keeps the chains; practically never taken
}

__global__ void k_probe_fill(uint4 *p, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = make_uint4((unsigned)i, (unsigned)(i >> 32), 0x5bd1e995u, 0u);
}

}  // namespace

extern "C" int hpr_bounds_violations(int64_t *count)
{
    if (!count) {
        g_static_err = "hpr_bounds_violations: count is NULL";
        return HPR_ERR_ARG;
    }
#ifdef HPR_BOUNDS_CHECK
    unsigned long long v = 0;
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpyFromSymbol(&v, hprdev::g_bounds_violations, sizeof v) != cudaSuccess) {
        (void)cudaGetLastError();
        g_static_err = "hpr_bounds_violations: the counter could not be read";
        return HPR_ERR_CUDA;
    }
    *count = (int64_t)v;
#else
    *count = -1;
#endif
    return HPR_OK;
}

extern "C" int hpr_memory_probe(int64_t read_bytes, int64_t gather_len, void *cuda_stream, double *read_gbs,
                                double *gather_gps)
{
    if (read_bytes < (1 << 20) || read_bytes > ((int64_t)1 << 34) || gather_len < 1024 ||
        gather_len > ((int64_t)1 << 28) || (gather_len & (gather_len - 1)) != 0) {
        g_static_err = "hpr_memory_probe: read_bytes in [1 MiB, 16 GiB], gather_len a power of two in [2^10, 2^28]";
        return HPR_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0, l2 = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess) {
        (void)cudaGetLastError();
        g_static_err = "hpr_memory_probe: no CUDA device";
        return HPR_ERR_NO_DEVICE;
    }
    const int64_t nread = read_bytes / 16, nflush = std::max<int64_t>(4 * (int64_t)l2, (int64_t)1 << 28) / 16;
    uint4 *buf = nullptr, *flush = nullptr;
    double *gx = nullptr;
    unsigned long long *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = HPR_OK;
    auto ok = [&](cudaError_t e) {
        if (e != cudaSuccess && rc == HPR_OK) {
            rc = e == cudaErrorMemoryAllocation ? HPR_ERR_NOMEM : HPR_ERR_CUDA;
            g_static_err = "hpr_memory_probe: CUDA error";
        }
        return rc == HPR_OK;
    };
    if (ok(cudaMalloc((void **)&buf, (size_t)nread * 16)) && ok(cudaMalloc((void **)&flush, (size_t)nflush * 16)) &&
        ok(cudaMalloc((void **)&gx, (size_t)gather_len * 8)) && ok(cudaMalloc((void **)&out, 64)) &&
        ok(cudaEventCreate(&e0)) && ok(cudaEventCreate(&e1))) {
        k_probe_fill<<<sms * 8, 256, 0, s>>>(buf, nread);
        k_probe_fill<<<sms * 8, 256, 0, s>>>(reinterpret_cast<uint4 *>(gx), gather_len / 2);
        float best_r = 1e30f, best_g = 1e30f;
        const int rounds = 64;
        k_probe_fill<<<sms * 8, 256, 0, s>>>(flush, nflush);
        for (int r = 0; r < 6 && rc == HPR_OK; ++r) {
            // evict buf from L2 by reading a buffer of 4x its size (reads leave clean lines, so
            // the timed stream pays no write-backs)
            k_probe_read<<<sms * 8, 256, 0, s>>>(flush, nflush, reinterpret_cast<unsigned *>(out));
            ok(cudaEventRecord(e0, s));
            k_probe_read<<<sms * 8, 256, 0, s>>>(buf, nread, reinterpret_cast<unsigned *>(out));
            ok(cudaEventRecord(e1, s));
            ok(cudaEventSynchronize(e1));
            float ms = 0.f;
            ok(cudaEventElapsedTime(&ms, e0, e1));
            if (r > 0) best_r = std::min(best_r, ms);                      // the first run warms up
            ok(cudaEventRecord(e0, s));                                     // gathers: x stays in L2
            k_probe_gather<<<sms * 8, 256, 0, s>>>(gx, (uint32_t)(gather_len - 1), rounds, out);
            ok(cudaEventRecord(e1, s));
            ok(cudaEventSynchronize(e1));
            ok(cudaEventElapsedTime(&ms, e0, e1));
            if (r > 0) best_g = std::min(best_g, ms);
        }
        ok(cudaGetLastError());
        if (rc == HPR_OK) {
            if (read_gbs) *read_gbs = (double)nread * 16.0 / (best_r * 1e-3) / 1e9;
            if (gather_gps) *gather_gps = (double)sms * 8 * 256 * rounds * 8 / (best_g * 1e-3) / 1e9;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    for (void *p : {(void *)buf, (void *)flush, (void *)gx, (void *)out})
        if (p) cudaFree(p);
    return rc;
}

// FP64 warp instructions per second of the whole GPU (DFMA with all 32 lanes active)
extern "C" int hpr_fp64_probe(void *cuda_stream, double *warp_ginst_per_s)
{
    if (!warp_ginst_per_s) {
        g_static_err = "hpr_fp64_probe: warp_ginst_per_s is NULL";
        return HPR_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        (void)cudaGetLastError();
        g_static_err = "hpr_fp64_probe: no CUDA device";
        return HPR_ERR_NO_DEVICE;
    }
    double *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = HPR_OK;
    auto ok = [&](cudaError_t e) {
        if (e != cudaSuccess && rc == HPR_OK) {
            rc = e == cudaErrorMemoryAllocation ? HPR_ERR_NOMEM : HPR_ERR_CUDA;
            g_static_err = "hpr_fp64_probe: CUDA error";
        }
        return rc == HPR_OK;
    };
    const int rounds = 2048, grid = sms * 8;
    float best = 1e30f;
    if (ok(cudaMalloc((void **)&out, 64)) && ok(cudaEventCreate(&e0)) && ok(cudaEventCreate(&e1))) {
        for (int r = 0; r < 4 && rc == HPR_OK; ++r) {
            ok(cudaEventRecord(e0, s));
            k_probe_fp64<<<grid, 256, 0, s>>>(rounds, out);
            ok(cudaEventRecord(e1, s));
            ok(cudaEventSynchronize(e1));
            float ms = 0.f;
            ok(cudaEventElapsedTime(&ms, e0, e1));
            if (r > 0) best = std::min(best, ms);                           // the first run warms up
        }
        ok(cudaGetLastError());
        if (rc == HPR_OK) *warp_ginst_per_s = (double)grid * (256 / 32) * rounds * 8 / (best * 1e-3) / 1e9;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) cudaFree(out);
    return rc;
}
