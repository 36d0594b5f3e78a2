// The sigma policy network: host side of its inference, gradient and training kernels.
// Part of the hpr_api.cu translation unit (included once, at its end, so that the kernels
// of hpr_device.cuh are defined once and the file-local helpers are shared).
#pragma once

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
