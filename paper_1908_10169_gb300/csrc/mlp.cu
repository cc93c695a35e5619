// The learned skip's classifier: training (Adam on FP32 master weights; forward and backward
// passes at the FP16-rounded weights with FP32 accumulation), inference over sample arrays,
// the loss gradient (for checks), installing a model on a context, and sample recording.
//
// Every reduction runs in a fixed order (per-sample work in one warp, parameter gradients as
// per-chunk sums in sample order, chunk sums added in chunk order), so a given seed always
// gives the same model.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "dev_common.cuh"
#include "mlp.cuh"

namespace {

constexpr int SPB = 16;   // samples per CTA in the forward/backward kernel (one per warp)
constexpr int NCH = 8;    // sample chunks of the parameter-gradient kernel

// per-feature mean and standard deviation over n samples (two passes, FP64 sums)
__global__ void __launch_bounds__(256) mlp_norm_kernel(const float *x, int64_t n, float *norm) {
    __shared__ double red[256];
    const int k = blockIdx.x, tid = threadIdx.x;
    double s = 0.0;
    for (int64_t i = tid; i < n; i += 256) s += (double)x[i * MF + k];
    red[tid] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (tid < o) red[tid] += red[tid + o];
        __syncthreads();
    }
    const double mean = red[0] / (double)(n > 0 ? n : 1);
    __syncthreads();
    double v = 0.0;
    for (int64_t i = tid; i < n; i += 256) {
        const double d = (double)x[i * MF + k] - mean;
        v += d * d;
    }
    red[tid] = v;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (tid < o) red[tid] += red[tid + o];
        __syncthreads();
    }
    if (tid == 0) {
        const double sd = sqrt(red[0] / (double)(n > 0 ? n : 1));
        norm[MO_MEAN + k] = (float)mean;
        norm[MO_STD + k] = sd > 1e-6 ? (float)sd : 1.f;
    }
}

struct BatchBufs {
    int64_t *idx;      // B sample indices
    float *H1, *H2;    // B x MH activations (after ReLU)
    float *DH1, *DH2;  // B x MH gradients with respect to the pre-activations
    float *DZ;         // B
    float *LOSS;       // B
};

// Forward and backward pass of B samples, one warp per sample; lanes own hidden units
// (lane, lane + 32).  Sample s of the batch is x[idx[s]], drawn with replacement from a
// counter-based hash of (seed, step, s) unless `identity` (then s itself).
__global__ void __launch_bounds__(SPB * 32) mlp_fwdbwd_kernel(const float *x, const float *y, int64_t n, int B,
                                                             const __half *w, const float *norm, uint64_t seed,
                                                             int64_t step, int identity, float invB, BatchBufs bb) {
    __shared__ float sW1[MH * MF], sW2[MH * MH], sb1[MH], sb2[MH], sw3[MH], sb3, snorm[2 * MF];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < MH * MF; i += SPB * 32) sW1[i] = mlp_w(w, MO_W1 + i);
    for (int i = tid; i < MH * MH; i += SPB * 32) sW2[i] = mlp_w(w, MO_W2 + i);
    for (int i = tid; i < MH; i += SPB * 32) {
        sb1[i] = mlp_w(w, MO_B1 + i);
        sb2[i] = mlp_w(w, MO_B2 + i);
        sw3[i] = mlp_w(w, MO_W3 + i);
    }
    if (tid < 2 * MF) snorm[tid] = norm[tid];
    if (tid == 0) sb3 = mlp_w(w, MO_B3);
    __syncthreads();
    const int s = blockIdx.x * SPB + warp;
    if (s >= B) return;
    const int64_t i = identity ? (int64_t)s : (int64_t)(mix64(seed ^ mix64((uint64_t)step * 0x100000001ULL + (uint64_t)s)) % (uint64_t)n);
    if (lane == 0) bb.idx[s] = i;
    const float xs = lane < MF ? mlp_std(snorm, lane, x[i * MF + lane]) : 0.f;
    const int u0 = lane, u1 = lane + 32;
    // layer 1
    float a0 = sb1[u0], a1 = sb1[u1];
    for (int k = 0; k < MF; ++k) {
        const float xk = __shfl_sync(FULL_MASK, xs, k);
        a0 = fmaf(sW1[u0 * MF + k], xk, a0);
        a1 = fmaf(sW1[u1 * MF + k], xk, a1);
    }
    const float h1a = fmaxf(a0, 0.f), h1b = fmaxf(a1, 0.f);
    // layer 2
    float c0 = sb2[u0], c1 = sb2[u1];
    for (int k = 0; k < MH; ++k) {
        const float hk = __shfl_sync(FULL_MASK, k < 32 ? h1a : h1b, k & 31);
        c0 = fmaf(sW2[u0 * MH + k], hk, c0);
        c1 = fmaf(sW2[u1 * MH + k], hk, c1);
    }
    const float h2a = fmaxf(c0, 0.f), h2b = fmaxf(c1, 0.f);
    // output, in unit order (the same sum as the sequential inference)
    float z = sb3;
    for (int u = 0; u < MH; ++u) z = fmaf(sw3[u], __shfl_sync(FULL_MASK, u < 32 ? h2a : h2b, u & 31), z);
    // binary cross-entropy of the logit, mean over the batch
    const float lab = y[i];
    const float p = 1.f / (1.f + expf(-z));
    const float dz = (p - lab) * invB;
    const float d2a = h2a > 0.f ? dz * sw3[u0] : 0.f, d2b = h2b > 0.f ? dz * sw3[u1] : 0.f;
    float e0 = 0.f, e1 = 0.f;
    for (int u = 0; u < MH; ++u) {
        const float du = __shfl_sync(FULL_MASK, u < 32 ? d2a : d2b, u & 31);
        e0 = fmaf(sW2[u * MH + u0], du, e0);
        e1 = fmaf(sW2[u * MH + u1], du, e1);
    }
    const float d1a = h1a > 0.f ? e0 : 0.f, d1b = h1b > 0.f ? e1 : 0.f;
    const int64_t o = (int64_t)s * MH;
    bb.H1[o + u0] = h1a; bb.H1[o + u1] = h1b;
    bb.H2[o + u0] = h2a; bb.H2[o + u1] = h2b;
    bb.DH1[o + u0] = d1a; bb.DH1[o + u1] = d1b;
    bb.DH2[o + u0] = d2a; bb.DH2[o + u1] = d2b;
    if (lane == 0) {
        bb.DZ[s] = dz;
        bb.LOSS[s] = fmaxf(z, 0.f) - z * lab + log1pf(expf(-fabsf(z)));
    }
}

// Parameter gradients: thread per (weight, sample chunk), samples in increasing order.
__global__ void __launch_bounds__(128) mlp_wgrad_kernel(const float *x, const float *norm, int B, BatchBufs bb,
                                                        float *partial) {
    const int p = blockIdx.x * 128 + threadIdx.x;  // weight index (model index - 2F)
    const int c = blockIdx.y;
    if (p >= MW) return;
    const int s0 = (int)((int64_t)B * c / NCH), s1 = (int)((int64_t)B * (c + 1) / NCH);
    const int m = p + 2 * MF;
    float acc = 0.f;
    if (m < MO_B1) {  // W1[u][k]
        const int u = (m - MO_W1) / MF, k = (m - MO_W1) % MF;
        const float mean = norm[MO_MEAN + k], sd = norm[MO_STD + k];
        for (int s = s0; s < s1; ++s) acc = fmaf(bb.DH1[(int64_t)s * MH + u], (x[bb.idx[s] * MF + k] - mean) / sd, acc);
    } else if (m < MO_W2) {  // b1[u]
        const int u = m - MO_B1;
        for (int s = s0; s < s1; ++s) acc += bb.DH1[(int64_t)s * MH + u];
    } else if (m < MO_B2) {  // W2[u][k]
        const int u = (m - MO_W2) / MH, k = (m - MO_W2) % MH;
        for (int s = s0; s < s1; ++s) acc = fmaf(bb.DH2[(int64_t)s * MH + u], bb.H1[(int64_t)s * MH + k], acc);
    } else if (m < MO_W3) {  // b2[u]
        const int u = m - MO_B2;
        for (int s = s0; s < s1; ++s) acc += bb.DH2[(int64_t)s * MH + u];
    } else if (m < MO_B3) {  // w3[u]
        const int u = m - MO_W3;
        for (int s = s0; s < s1; ++s) acc = fmaf(bb.DZ[s], bb.H2[(int64_t)s * MH + u], acc);
    } else {  // b3
        for (int s = s0; s < s1; ++s) acc += bb.DZ[s];
    }
    partial[(int64_t)c * MW + p] = acc;
}

// Adam step on the FP32 master weights; the FP16 copy is what the passes use.
__global__ void __launch_bounds__(256) mlp_adam_kernel(const float *partial, float *master, float *mom, float *vel,
                                                       __half *w, float lr, float bc1, float bc2) {
    const int p = blockIdx.x * 256 + threadIdx.x;
    if (p >= MW) return;
    float g = 0.f;
    for (int c = 0; c < NCH; ++c) g += partial[(int64_t)c * MW + p];
    const float m = 0.9f * mom[p] + 0.1f * g;
    const float v = 0.999f * vel[p] + 0.001f * g * g;
    mom[p] = m;
    vel[p] = v;
    const float mw = master[p] - lr * (m / bc1) / (sqrtf(v / bc2) + 1e-8f);
    master[p] = mw;
    w[p] = __float2half_rn(mw);
}

__global__ void __launch_bounds__(128) mlp_forward_kernel(const float *x, int64_t n, const __half *w,
                                                          const float *norm, float *logits) {
    const int64_t i = (int64_t)blockIdx.x * 128 + threadIdx.x;
    if (i >= n) return;
    float xs[MF];
#pragma unroll
    for (int k = 0; k < MF; ++k) xs[k] = mlp_std(norm, k, x[i * MF + k]);
    logits[i] = mlp_logit_seq(xs, w);
}

// Device copies of a host model: FP32 normalisation, FP16 weights.
struct DevModel {
    float *norm = nullptr;
    __half *w = nullptr;
    ~DevModel() {
        dev_free(norm);
        dev_free(w);
    }
};

cudaError_t upload_model(const float *model, DevModel &dm, cudaStream_t st) {
    cudaError_t e;
    if ((e = dev_alloc(&dm.norm, 2 * MF)) != cudaSuccess || (e = dev_alloc(&dm.w, MW)) != cudaSuccess) return e;
    std::vector<__half> h(MW);
    for (int i = 0; i < MW; ++i) h[i] = __float2half_rn(model[2 * MF + i]);
    if ((e = cudaMemcpyAsync(dm.norm, model, 2 * MF * sizeof(float), cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(dm.w, h.data(), MW * sizeof(__half), cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    return cudaStreamSynchronize(st);  // h goes out of scope
}

bool model_ok(const float *model) {
    for (int i = 0; i < MO_N; ++i)
        if (!std::isfinite(model[i])) return false;
    for (int k = 0; k < MF; ++k)
        if (!(model[MO_STD + k] > 0.f)) return false;
    return true;
}

// device copy of caller samples (host or device memory)
template <class T>
cudaError_t stage(const T *src, int64_t count, T **dst, cudaStream_t st) {
    cudaError_t e = dev_alloc(dst, count);
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(*dst, src, (size_t)count * sizeof(T), cudaMemcpyDefault, st);
}

struct Scratch {
    BatchBufs bb{};
    float *partial = nullptr;
    cudaError_t alloc(int B) {
        cudaError_t e;
        if ((e = dev_alloc(&bb.idx, B)) != cudaSuccess || (e = dev_alloc(&bb.H1, (int64_t)B * MH)) != cudaSuccess ||
            (e = dev_alloc(&bb.H2, (int64_t)B * MH)) != cudaSuccess || (e = dev_alloc(&bb.DH1, (int64_t)B * MH)) != cudaSuccess ||
            (e = dev_alloc(&bb.DH2, (int64_t)B * MH)) != cudaSuccess || (e = dev_alloc(&bb.DZ, B)) != cudaSuccess ||
            (e = dev_alloc(&bb.LOSS, B)) != cudaSuccess || (e = dev_alloc(&partial, (int64_t)NCH * MW)) != cudaSuccess)
            return e;
        return cudaSuccess;
    }
    ~Scratch() {
        dev_free(bb.idx); dev_free(bb.H1); dev_free(bb.H2); dev_free(bb.DH1); dev_free(bb.DH2);
        dev_free(bb.DZ); dev_free(bb.LOSS); dev_free(partial);
    }
};

bilu_status check_ctx(bilu_ctx *c) {
    if (!c) return BILU_ERR_ARG;
    c->err.clear();
    BILU_CUDA(c, cudaSetDevice(c->device));
    return BILU_OK;
}

}  // namespace

void mlp_free(bilu_ctx *c) {
    dev_free(c->d_mlp_norm);
    if (c->d_mlp_w) cudaFree(c->d_mlp_w);
    c->d_mlp_w = nullptr;
    dev_free(c->d_rec_x);
    dev_free(c->d_rec_y);
    dev_free(c->d_rec_tag);
    dev_free(c->d_rec_count);
    dev_free(c->d_featL);
    dev_free(c->d_featU);
    c->rec_cap = 0;
    c->feat_cap = 0;
}

extern "C" {

bilu_status bilu_mlp_train(bilu_ctx *c, const float *x, const float *y, int64_t n, const bilu_mlp_train_cfg *cfg,
                           float *model, double *final_loss) {
    bilu_status st0 = check_ctx(c);
    if (st0 != BILU_OK) return st0;
    if (!x || !y || !cfg || !model || n < 1) return set_err(c, BILU_ERR_ARG, "bilu_mlp_train: bad arguments");
    if (cfg->epochs < 0 || cfg->batch < 1 || cfg->batch > 65536 || !(cfg->lr > 0.f))
        return set_err(c, BILU_ERR_ARG, "bilu_mlp_train: bad configuration");
    const cudaStream_t st = c->stream;
    const int B = cfg->batch;
    float *dx = nullptr, *dy = nullptr, *norm = nullptr, *master = nullptr, *mom = nullptr, *vel = nullptr;
    __half *w = nullptr;
    Scratch sc;
    auto cleanup = [&]() {
        dev_free(dx); dev_free(dy); dev_free(norm); dev_free(master); dev_free(mom); dev_free(vel); dev_free(w);
    };
    cudaError_t e;
    if ((e = stage(x, n * MF, &dx, st)) != cudaSuccess || (e = stage(y, n, &dy, st)) != cudaSuccess ||
        (e = dev_alloc(&norm, 2 * MF)) != cudaSuccess || (e = dev_alloc(&master, MW)) != cudaSuccess ||
        (e = dev_alloc(&mom, MW)) != cudaSuccess || (e = dev_alloc(&vel, MW)) != cudaSuccess ||
        (e = dev_alloc(&w, MW)) != cudaSuccess || (e = sc.alloc(std::max<int64_t>(B, std::min<int64_t>(n, 65536)))) != cudaSuccess) {
        cleanup();
        return e == cudaErrorMemoryAllocation ? set_err(c, BILU_ERR_OOM, "bilu_mlp_train: allocation failed")
                                              : cuda_err(c, e, "bilu_mlp_train staging");
    }
    mlp_norm_kernel<<<MF, 256, 0, st>>>(dx, n, norm);
    c->launches += 1;
    // initial weights: uniform in +-1/sqrt(fan-in) from a counter-based hash, biases 0
    std::vector<float> hm(MW, 0.f);
    std::vector<__half> hh(MW);
    for (int p = 0; p < MW; ++p) {
        const int mi = p + 2 * MF;
        float bound = 0.f;
        if (mi >= MO_W1 && mi < MO_B1) bound = 1.f / std::sqrt((float)MF);
        else if (mi >= MO_W2 && mi < MO_B2) bound = 1.f / std::sqrt((float)MH);
        else if (mi >= MO_W3 && mi < MO_B3) bound = 1.f / std::sqrt((float)MH);
        const double u = (double)(mix64(cfg->seed ^ mix64(0xA5A5A5A5ULL + (uint64_t)p)) >> 11) * (1.0 / 9007199254740992.0);
        hm[p] = __half2float(__float2half_rn((float)((2.0 * u - 1.0) * bound)));
        hh[p] = __float2half_rn(hm[p]);
    }
    cudaMemcpyAsync(master, hm.data(), MW * sizeof(float), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(w, hh.data(), MW * sizeof(__half), cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(mom, 0, MW * sizeof(float), st);
    cudaMemsetAsync(vel, 0, MW * sizeof(float), st);
    const int64_t steps_per_epoch = (n + B - 1) / B;
    const int64_t steps = steps_per_epoch * cfg->epochs;
    double b1t = 1.0, b2t = 1.0;
    for (int64_t t = 0; t < steps; ++t) {
        mlp_fwdbwd_kernel<<<(B + SPB - 1) / SPB, SPB * 32, 0, st>>>(dx, dy, n, B, w, norm, cfg->seed, t, 0, 1.f / (float)B, sc.bb);
        mlp_wgrad_kernel<<<dim3((MW + 127) / 128, NCH), 128, 0, st>>>(dx, norm, B, sc.bb, sc.partial);
        b1t *= 0.9;
        b2t *= 0.999;
        mlp_adam_kernel<<<(MW + 255) / 256, 256, 0, st>>>(sc.partial, master, mom, vel, w, cfg->lr, (float)(1.0 - b1t), (float)(1.0 - b2t));
        c->launches += 3;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) { cleanup(); return cuda_err(c, e, "bilu_mlp_train kernels"); }
    // the model: normalisation and the FP16-rounded weights, as FP32
    std::vector<float> nrm(2 * MF);
    cudaMemcpyAsync(nrm.data(), norm, 2 * MF * sizeof(float), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(hh.data(), w, MW * sizeof(__half), cudaMemcpyDeviceToHost, st);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) { cleanup(); return cuda_err(c, e, "bilu_mlp_train"); }
    for (int k = 0; k < 2 * MF; ++k) model[k] = nrm[k];
    for (int p = 0; p < MW; ++p) model[2 * MF + p] = __half2float(hh[p]);
    if (final_loss) {
        // mean cross-entropy over all samples, in chunks of the scratch size
        const int64_t chunk = std::min<int64_t>(n, 65536);
        std::vector<float> loss(chunk);
        double sum = 0.0;
        for (int64_t s0 = 0; s0 < n; s0 += chunk) {
            const int cnt = (int)std::min<int64_t>(chunk, n - s0);
            mlp_fwdbwd_kernel<<<(cnt + SPB - 1) / SPB, SPB * 32, 0, st>>>(dx + s0 * MF, dy + s0, cnt, cnt, w, norm, 0, 0, 1,
                                                                        1.f / (float)cnt, sc.bb);
            c->launches += 1;
            cudaMemcpyAsync(loss.data(), sc.bb.LOSS, cnt * sizeof(float), cudaMemcpyDeviceToHost, st);
            if ((e = cudaStreamSynchronize(st)) != cudaSuccess) { cleanup(); return cuda_err(c, e, "bilu_mlp_train loss"); }
            for (int i = 0; i < cnt; ++i) sum += loss[i];
        }
        *final_loss = sum / (double)n;
    }
    cleanup();
    return BILU_OK;
}

bilu_status bilu_mlp_forward(bilu_ctx *c, const float *model, const float *x, int64_t n, float *logits) {
    bilu_status st0 = check_ctx(c);
    if (st0 != BILU_OK) return st0;
    if (!model || !x || !logits || n < 0) return set_err(c, BILU_ERR_ARG, "bilu_mlp_forward: bad arguments");
    if (!model_ok(model)) return set_err(c, BILU_ERR_ARG, "bilu_mlp_forward: model has non-finite entries or std <= 0");
    if (n == 0) return BILU_OK;
    DevModel dm;
    float *dx = nullptr, *dl = nullptr;
    cudaError_t e;
    if ((e = upload_model(model, dm, c->stream)) != cudaSuccess || (e = stage(x, n * MF, &dx, c->stream)) != cudaSuccess ||
        (e = dev_alloc(&dl, n)) != cudaSuccess) {
        dev_free(dx); dev_free(dl);
        return cuda_err(c, e, "bilu_mlp_forward staging");
    }
    mlp_forward_kernel<<<(unsigned)((n + 127) / 128), 128, 0, c->stream>>>(dx, n, dm.w, dm.norm, dl);
    c->launches += 1;
    e = cudaMemcpyAsync(logits, dl, n * sizeof(float), cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dev_free(dx); dev_free(dl);
    if (e != cudaSuccess) return cuda_err(c, e, "bilu_mlp_forward");
    return BILU_OK;
}

bilu_status bilu_mlp_grad(bilu_ctx *c, const float *model, const float *x, const float *y, int64_t n, float *grad) {
    bilu_status st0 = check_ctx(c);
    if (st0 != BILU_OK) return st0;
    if (!model || !x || !y || !grad || n < 1 || n > 65536) return set_err(c, BILU_ERR_ARG, "bilu_mlp_grad: bad arguments (1 <= n <= 65536)");
    if (!model_ok(model)) return set_err(c, BILU_ERR_ARG, "bilu_mlp_grad: model has non-finite entries or std <= 0");
    DevModel dm;
    float *dx = nullptr, *dy = nullptr;
    Scratch sc;
    cudaError_t e;
    if ((e = upload_model(model, dm, c->stream)) != cudaSuccess || (e = stage(x, n * MF, &dx, c->stream)) != cudaSuccess ||
        (e = stage(y, n, &dy, c->stream)) != cudaSuccess || (e = sc.alloc((int)n)) != cudaSuccess) {
        dev_free(dx); dev_free(dy);
        return cuda_err(c, e, "bilu_mlp_grad staging");
    }
    mlp_fwdbwd_kernel<<<(unsigned)((n + SPB - 1) / SPB), SPB * 32, 0, c->stream>>>(dx, dy, n, (int)n, dm.w, dm.norm, 0, 0, 1,
                                                                                 1.f / (float)n, sc.bb);
    mlp_wgrad_kernel<<<dim3((MW + 127) / 128, NCH), 128, 0, c->stream>>>(dx, dm.norm, (int)n, sc.bb, sc.partial);
    c->launches += 2;
    std::vector<float> part((size_t)NCH * MW);
    e = cudaMemcpyAsync(part.data(), sc.partial, part.size() * sizeof(float), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dev_free(dx); dev_free(dy);
    if (e != cudaSuccess) return cuda_err(c, e, "bilu_mlp_grad");
    for (int k = 0; k < 2 * MF; ++k) grad[k] = 0.f;
    for (int p = 0; p < MW; ++p) {
        float g = 0.f;
        for (int ch = 0; ch < NCH; ++ch) g += part[(size_t)ch * MW + p];
        grad[2 * MF + p] = g;
    }
    return BILU_OK;
}

bilu_status bilu_set_skip_model(bilu_ctx *c, const float *model, double logit_hi) {
    bilu_status st0 = check_ctx(c);
    if (st0 != BILU_OK) return st0;
    if (!model || !std::isfinite(logit_hi)) return set_err(c, BILU_ERR_ARG, "bilu_set_skip_model: bad arguments");
    if (!model_ok(model)) return set_err(c, BILU_ERR_ARG, "bilu_set_skip_model: model has non-finite entries or std <= 0");
    dev_free(c->d_mlp_norm);
    if (c->d_mlp_w) cudaFree(c->d_mlp_w);
    c->d_mlp_w = nullptr;
    __half *w = nullptr;
    if (dev_alloc(&c->d_mlp_norm, 2 * MF) != cudaSuccess || dev_alloc(&w, MW) != cudaSuccess) {
        dev_free(c->d_mlp_norm);
        dev_free(w);
        return set_err(c, BILU_ERR_OOM, "bilu_set_skip_model: allocation failed");
    }
    c->d_mlp_w = w;
    std::vector<__half> h(MW);
    for (int i = 0; i < MW; ++i) h[i] = __float2half_rn(model[2 * MF + i]);
    BILU_CUDA(c, cudaMemcpyAsync(c->d_mlp_norm, model, 2 * MF * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    BILU_CUDA(c, cudaMemcpyAsync(w, h.data(), MW * sizeof(__half), cudaMemcpyHostToDevice, c->stream));
    BILU_CUDA(c, cudaStreamSynchronize(c->stream));
    c->mlp_logit_hi = logit_hi;
    return BILU_OK;
}

bilu_status bilu_record_samples(bilu_ctx *c, int64_t capacity, double rate, uint64_t seed) {
    bilu_status st0 = check_ctx(c);
    if (st0 != BILU_OK) return st0;
    if (capacity < 0 || !(rate >= 0.0 && rate <= 1.0)) return set_err(c, BILU_ERR_ARG, "bilu_record_samples: bad arguments");
    dev_free(c->d_rec_x);
    dev_free(c->d_rec_y);
    dev_free(c->d_rec_tag);
    dev_free(c->d_rec_count);
    c->rec_cap = 0;
    c->rec_base = 0;
    if (capacity == 0) {
        dev_free(c->d_featL);
        dev_free(c->d_featU);
        c->feat_cap = 0;
        return BILU_OK;
    }
    if (dev_alloc(&c->d_rec_x, capacity * MF) != cudaSuccess || dev_alloc(&c->d_rec_y, capacity) != cudaSuccess ||
        dev_alloc(&c->d_rec_tag, capacity) != cudaSuccess || dev_alloc(&c->d_rec_count, 1) != cudaSuccess) {
        dev_free(c->d_rec_x); dev_free(c->d_rec_y); dev_free(c->d_rec_tag); dev_free(c->d_rec_count);
        return set_err(c, BILU_ERR_OOM, "bilu_record_samples: allocation failed");
    }
    BILU_CUDA(c, cudaMemsetAsync(c->d_rec_count, 0, sizeof(unsigned long long), c->stream));
    BILU_CUDA(c, cudaStreamSynchronize(c->stream));
    c->rec_cap = capacity;
    c->rec_thresh = rate >= 1.0 ? 0xffffffffu : (uint32_t)(rate * 4294967296.0);
    c->rec_seed = seed;
    return BILU_OK;
}

bilu_status bilu_get_samples(bilu_ctx *c, float *x, float *y, int64_t *tags, int64_t cap, int64_t *count) {
    bilu_status st0 = check_ctx(c);
    if (st0 != BILU_OK) return st0;
    if (!count || cap < 0 || (cap > 0 && (!x || !y))) return set_err(c, BILU_ERR_ARG, "bilu_get_samples: bad arguments");
    if (c->rec_cap == 0) {
        *count = 0;
        return BILU_OK;
    }
    unsigned long long held = 0;
    BILU_CUDA(c, cudaMemcpyAsync(&held, c->d_rec_count, sizeof(held), cudaMemcpyDeviceToHost, c->stream));
    BILU_CUDA(c, cudaStreamSynchronize(c->stream));
    const int64_t have = std::min<int64_t>((int64_t)held, c->rec_cap);
    const int64_t m = std::min<int64_t>(have, cap);
    if (m > 0) {
        BILU_CUDA(c, cudaMemcpyAsync(x, c->d_rec_x, (size_t)m * MF * sizeof(float), cudaMemcpyDefault, c->stream));
        BILU_CUDA(c, cudaMemcpyAsync(y, c->d_rec_y, (size_t)m * sizeof(float), cudaMemcpyDefault, c->stream));
        if (tags)
            BILU_CUDA(c, cudaMemcpyAsync(tags, c->d_rec_tag, (size_t)m * sizeof(int64_t), cudaMemcpyDefault, c->stream));
        BILU_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    *count = have;
    return BILU_OK;
}

}  // extern "C"
