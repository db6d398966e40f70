// A small 3D U-Net with hand-written forward, backward and Adam kernels, used
// to predict the per-step head / temperature increments as Krylov initial
// guesses.  Weights are held as FP32 masters and used in BF16 in the forward
// and data-gradient convolutions; every accumulation is FP32 and every
// reduction runs in a fixed order (bitwise reproducible).
//
//   e1 = relu(conv3(x;  Cin -> C1))        p1 = avgpool2(e1)
//   e2 = relu(conv3(p1; C1 -> C2))         u2 = upsample2(e2)
//   d1 = relu(conv3([e1, u2]; C1+C2 -> C1))
//   y  = conv1(d1; C1 -> Cout)            loss = mean (y - target)^2
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <string>
#include <vector>

#include "ht.h"

namespace {

constexpr int C1 = 16, C2 = 32;       // channel widths of the two levels

struct Vol {
    int D, H, W;
    __host__ __device__ int n() const { return D * H * W; }
};

__device__ __forceinline__ float ldx(const float* x, const Vol& v, int z, int y, int w) {
    return (z < 0 || z >= v.D || y < 0 || y >= v.H || w < 0 || w >= v.W) ? 0.f : x[(z * v.H + y) * v.W + w];
}

// ---- convolution forward: one thread per voxel, all CO outputs in registers
template <int CO, int K>
__global__ void __launch_bounds__(128) conv_fwd_kernel(const float* __restrict__ in, int ci_n, const Vol v,
                                                       const __nv_bfloat16* __restrict__ w,
                                                       const float* __restrict__ bias, float* __restrict__ pre,
                                                       float* __restrict__ post) {
    extern __shared__ float ws[];   // [CO][ci][K]
    const int nw = CO * ci_n * K;
    for (int i = threadIdx.x; i < nw; i += blockDim.x) ws[i] = __bfloat162float(w[i]);
    __syncthreads();
    const int n = v.n();
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int xw = p % v.W, t = p / v.W, yh = t % v.H, zd = t / v.H;
        float acc[CO];
#pragma unroll
        for (int o = 0; o < CO; ++o) acc[o] = bias[o];
        for (int c = 0; c < ci_n; ++c) {
            const float* xc = in + (size_t)c * n;
#pragma unroll
            for (int tp = 0; tp < K; ++tp) {
                const int dz = K == 1 ? 0 : tp / 9 - 1, dy = K == 1 ? 0 : (tp / 3) % 3 - 1, dx = K == 1 ? 0 : tp % 3 - 1;
                const float xv = ldx(xc, v, zd + dz, yh + dy, xw + dx);
#pragma unroll
                for (int o = 0; o < CO; ++o) acc[o] = fmaf(ws[(o * ci_n + c) * K + tp], xv, acc[o]);
            }
        }
#pragma unroll
        for (int o = 0; o < CO; ++o) {
            if (pre) pre[(size_t)o * n + p] = acc[o];
            if (post) post[(size_t)o * n + p] = fmaxf(acc[o], 0.f);
        }
    }
}

// ---- convolution data gradient: g_in[ci][p] = sum_co sum_t w[co][ci][t] g_out[co][p - d_t]
template <int CI, int K>
__global__ void __launch_bounds__(128) conv_bwd_data_kernel(const float* __restrict__ gout, int co_n, const Vol v,
                                                            const __nv_bfloat16* __restrict__ w,
                                                            float* __restrict__ gin) {
    extern __shared__ float ws[];   // [co][CI][K]
    const int nw = co_n * CI * K;
    for (int i = threadIdx.x; i < nw; i += blockDim.x) ws[i] = __bfloat162float(w[i]);
    __syncthreads();
    const int n = v.n();
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int xw = p % v.W, t = p / v.W, yh = t % v.H, zd = t / v.H;
        float acc[CI];
#pragma unroll
        for (int c = 0; c < CI; ++c) acc[c] = 0.f;
        for (int o = 0; o < co_n; ++o) {
            const float* go = gout + (size_t)o * n;
#pragma unroll
            for (int tp = 0; tp < K; ++tp) {
                const int dz = K == 1 ? 0 : tp / 9 - 1, dy = K == 1 ? 0 : (tp / 3) % 3 - 1, dx = K == 1 ? 0 : tp % 3 - 1;
                const float gv = ldx(go, v, zd - dz, yh - dy, xw - dx);
#pragma unroll
                for (int c = 0; c < CI; ++c) acc[c] = fmaf(ws[(o * CI + c) * K + tp], gv, acc[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < CI; ++c) gin[(size_t)c * n + p] = acc[c];
    }
}

__device__ __forceinline__ float block_sum_f(float v, float* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    v = (threadIdx.x < (blockDim.x >> 5)) ? sh[lane] : 0.f;
    if (wid == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

// ---- weight gradient: one CTA per (co, ci), K accumulators per thread
template <int K>
__global__ void __launch_bounds__(256) conv_bwd_weight_kernel(const float* __restrict__ in, int ci_n,
                                                              const float* __restrict__ gout, const Vol v,
                                                              float* __restrict__ gw) {
    __shared__ float sh[32];
    const int o = blockIdx.x / ci_n, c = blockIdx.x % ci_n;
    const int n = v.n();
    const float* xc = in + (size_t)c * n;
    const float* go = gout + (size_t)o * n;
    float acc[K];
#pragma unroll
    for (int tp = 0; tp < K; ++tp) acc[tp] = 0.f;
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
        const float g = go[p];
        const int xw = p % v.W, t = p / v.W, yh = t % v.H, zd = t / v.H;
#pragma unroll
        for (int tp = 0; tp < K; ++tp) {
            const int dz = K == 1 ? 0 : tp / 9 - 1, dy = K == 1 ? 0 : (tp / 3) % 3 - 1, dx = K == 1 ? 0 : tp % 3 - 1;
            acc[tp] = fmaf(g, ldx(xc, v, zd + dz, yh + dy, xw + dx), acc[tp]);
        }
    }
#pragma unroll
    for (int tp = 0; tp < K; ++tp) {
        const float s = block_sum_f(acc[tp], sh);
        if (threadIdx.x == 0) gw[(o * ci_n + c) * K + tp] = s;
    }
}

__global__ void bias_grad_kernel(const float* __restrict__ gout, int n, float* __restrict__ gb) {
    __shared__ float sh[32];
    const float* go = gout + (size_t)blockIdx.x * n;
    float s = 0.f;
    for (int p = threadIdx.x; p < n; p += blockDim.x) s += go[p];
    s = block_sum_f(s, sh);
    if (threadIdx.x == 0) gb[blockIdx.x] = s;
}

__global__ void relu_bwd_kernel(float* __restrict__ g, const float* __restrict__ pre, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        if (!(pre[i] > 0.f)) g[i] = 0.f;
}

// 2x2x2 mean pooling of C channels: fine v -> coarse
__global__ void pool_kernel(const float* __restrict__ in, int C, const Vol v, float* __restrict__ out) {
    const Vol c2{v.D / 2, v.H / 2, v.W / 2};
    const int nc = c2.n(), nf = v.n();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)C * nc;
         i += (long long)gridDim.x * blockDim.x) {
        const int ch = (int)(i / nc), p = (int)(i % nc);
        const int xw = p % c2.W, t = p / c2.W, yh = t % c2.H, zd = t / c2.H;
        const float* src = in + (size_t)ch * nf;
        float s = 0.f;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int d = 0; d < 2; ++d) s += src[((2 * zd + a) * v.H + 2 * yh + b) * v.W + 2 * xw + d];
        out[i] = 0.125f * s;
    }
}

// pooling backward (adds into gfine) and nearest upsampling (writes fine)
__global__ void pool_bwd_add_kernel(const float* __restrict__ gc, int C, const Vol v, float* __restrict__ gf) {
    const Vol c2{v.D / 2, v.H / 2, v.W / 2};
    const int nf = v.n(), nc = c2.n();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)C * nf;
         i += (long long)gridDim.x * blockDim.x) {
        const int ch = (int)(i / nf), p = (int)(i % nf);
        const int xw = p % v.W, t = p / v.W, yh = t % v.H, zd = t / v.H;
        gf[i] += 0.125f * gc[(size_t)ch * nc + ((zd / 2) * c2.H + yh / 2) * c2.W + xw / 2];
    }
}

__global__ void upsample_kernel(const float* __restrict__ coarse, int C, const Vol v, float* __restrict__ fine) {
    const Vol c2{v.D / 2, v.H / 2, v.W / 2};
    const int nf = v.n(), nc = c2.n();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)C * nf;
         i += (long long)gridDim.x * blockDim.x) {
        const int ch = (int)(i / nf), p = (int)(i % nf);
        const int xw = p % v.W, t = p / v.W, yh = t % v.H, zd = t / v.H;
        fine[i] = coarse[(size_t)ch * nc + ((zd / 2) * c2.H + yh / 2) * c2.W + xw / 2];
    }
}

__global__ void upsample_bwd_kernel(const float* __restrict__ gfine, int C, const Vol v, float* __restrict__ gc) {
    const Vol c2{v.D / 2, v.H / 2, v.W / 2};
    const int nf = v.n(), nc = c2.n();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)C * nc;
         i += (long long)gridDim.x * blockDim.x) {
        const int ch = (int)(i / nc), p = (int)(i % nc);
        const int xw = p % c2.W, t = p / c2.W, yh = t % c2.H, zd = t / c2.H;
        const float* src = gfine + (size_t)ch * nf;
        float s = 0.f;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int d = 0; d < 2; ++d) s += src[((2 * zd + a) * v.H + 2 * yh + b) * v.W + 2 * xw + d];
        gc[i] = s;
    }
}

// MSE: g = 2 (y - t) / N; per-block partial sums of (y - t)^2
__global__ void mse_kernel(const float* __restrict__ y, const float* __restrict__ t, long long n,
                           float* __restrict__ g, float* __restrict__ part) {
    __shared__ float sh[32];
    float s = 0.f;
    const float scale = 2.0f / (float)n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float d = y[i] - t[i];
        g[i] = scale * d;
        s = fmaf(d, d, s);
    }
    s = block_sum_f(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void adam_kernel(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ vv,
                            const float* __restrict__ g, int n, float lr, float b1, float b2, float c1, float c2,
                            float eps, __nv_bfloat16* __restrict__ wb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * vv[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    vv[i] = vi;
    const float th = theta[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    theta[i] = th;
    wb[i] = __float2bfloat16_rn(th);
}

__global__ void to_bf16_kernel(const float* __restrict__ a, __nv_bfloat16* __restrict__ b, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = __float2bfloat16_rn(a[i]);
}

}  // namespace

struct ht_unet {
    int cin = 4, cout = 2, device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int np = 0;
    int off[4][2];                 // weight / bias offsets of the four layers
    float *theta = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    __nv_bfloat16* wb = nullptr;   // BF16 copy of theta (weights and biases)
    float* wfp = nullptr;          // biases read in FP32 from theta
    // activations (sized for the largest grid seen)
    size_t cap = 0;
    float *a1 = nullptr, *cat = nullptr, *p1 = nullptr, *a2 = nullptr, *e2 = nullptr, *a3 = nullptr, *d1 = nullptr;
    float *y = nullptr, *gy = nullptr, *gd1 = nullptr, *gcat = nullptr, *ge2c = nullptr, *gp1 = nullptr, *ga1 = nullptr;
    float* lpart = nullptr;
    int step = 0;
    std::string err;
};

namespace {

int layer_ci(const ht_unet* u, int l) { return l == 0 ? u->cin : (l == 1 ? C1 : (l == 2 ? C1 + C2 : C1)); }
int layer_co(const ht_unet* u, int l) { return l == 0 ? C1 : (l == 1 ? C2 : (l == 2 ? C1 : u->cout)); }
int layer_k(int l) { return l == 3 ? 1 : 27; }

int ufail(ht_unet* u, int code, const char* msg) {
    if (u) u->err = msg;
    return code;
}

int ensure(ht_unet* u, const Vol& v) {
    const size_t n = (size_t)v.n();
    if (n <= u->cap) return HT_OK;
    float** bufs[] = {&u->a1, &u->cat, &u->p1, &u->a2, &u->e2, &u->a3, &u->d1, &u->y, &u->gy, &u->gd1,
                      &u->gcat, &u->ge2c, &u->gp1, &u->ga1};
    const size_t sizes[] = {C1 * n, (C1 + C2) * n, C1 * n / 8 + 8, C2 * n / 8 + 8, C2 * n / 8 + 8, C1 * n,
                            C1 * n, (size_t)u->cout * n, (size_t)u->cout * n, C1 * n, (C1 + C2) * n,
                            C2 * n / 8 + 8, C1 * n / 8 + 8, C1 * n};
    for (int i = 0; i < 14; ++i) {
        if (*bufs[i]) cudaFree(*bufs[i]);
        *bufs[i] = nullptr;
        if (cudaMalloc(bufs[i], sizes[i] * sizeof(float)) != cudaSuccess) return ufail(u, HT_ENOMEM, "activation alloc");
    }
    u->cap = n;
    return HT_OK;
}

int grid_for(long long n) {
    long long b = (n + 127) / 128;
    return (int)(b > 4096 ? 4096 : (b < 1 ? 1 : b));
}

template <int CO, int K>
void conv_fwd(ht_unet* u, int l, const float* in, const Vol& v, float* pre, float* post) {
    const int ci = layer_ci(u, l);
    const size_t smem = (size_t)CO * ci * K * sizeof(float);
    cudaFuncSetAttribute(conv_fwd_kernel<CO, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    conv_fwd_kernel<CO, K><<<grid_for(v.n()), 128, smem, u->stream>>>(in, ci, v, u->wb + u->off[l][0],
                                                                      u->theta + u->off[l][1], pre, post);
}

template <int CI, int K>
void conv_bwd_data(ht_unet* u, int l, const float* gout, const Vol& v, float* gin) {
    const int co = layer_co(u, l);
    const size_t smem = (size_t)co * CI * K * sizeof(float);
    cudaFuncSetAttribute(conv_bwd_data_kernel<CI, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    conv_bwd_data_kernel<CI, K><<<grid_for(v.n()), 128, smem, u->stream>>>(gout, co, v, u->wb + u->off[l][0], gin);
}

void conv_bwd_weight(ht_unet* u, int l, const float* in, const float* gout, const Vol& v) {
    const int ci = layer_ci(u, l), co = layer_co(u, l);
    if (layer_k(l) == 27)
        conv_bwd_weight_kernel<27><<<co * ci, 256, 0, u->stream>>>(in, ci, gout, v, u->grad + u->off[l][0]);
    else
        conv_bwd_weight_kernel<1><<<co * ci, 256, 0, u->stream>>>(in, ci, gout, v, u->grad + u->off[l][0]);
    bias_grad_kernel<<<co, 256, 0, u->stream>>>(gout, v.n(), u->grad + u->off[l][1]);
}

int forward(ht_unet* u, const float* x, const Vol& v) {
    const Vol vc{v.D / 2, v.H / 2, v.W / 2};
    float* e1 = u->cat;                        // the first C1 channels of the concatenation
    float* u2 = u->cat + (size_t)C1 * v.n();
    conv_fwd<C1, 27>(u, 0, x, v, u->a1, e1);
    pool_kernel<<<grid_for((long long)C1 * vc.n()), 128, 0, u->stream>>>(e1, C1, v, u->p1);
    conv_fwd<C2, 27>(u, 1, u->p1, vc, u->a2, u->e2);
    upsample_kernel<<<grid_for((long long)C2 * v.n()), 128, 0, u->stream>>>(u->e2, C2, v, u2);
    conv_fwd<C1, 27>(u, 2, u->cat, v, u->a3, u->d1);
    conv_fwd<2, 1>(u, 3, u->d1, v, u->y, nullptr);   // linear output layer
    return cudaGetLastError() == cudaSuccess ? HT_OK : ufail(u, HT_ECUDA, "forward launch failed");
}

// loss and gradients into u->grad (forward must have run)
int backward(ht_unet* u, const float* x, const float* target, const Vol& v, double* loss) {
    const Vol vc{v.D / 2, v.H / 2, v.W / 2};
    const long long ny = (long long)u->cout * v.n();
    const int G = grid_for(ny) > 1024 ? 1024 : grid_for(ny);
    mse_kernel<<<G, 128, 0, u->stream>>>(u->y, target, ny, u->gy, u->lpart);
    conv_bwd_weight(u, 3, u->d1, u->gy, v);
    conv_bwd_data<C1, 1>(u, 3, u->gy, v, u->gd1);
    relu_bwd_kernel<<<grid_for((long long)C1 * v.n()), 128, 0, u->stream>>>(u->gd1, u->a3, (long long)C1 * v.n());
    conv_bwd_weight(u, 2, u->cat, u->gd1, v);
    conv_bwd_data<C1 + C2, 27>(u, 2, u->gd1, v, u->gcat);
    float* ge1 = u->gcat;
    float* gu2 = u->gcat + (size_t)C1 * v.n();
    upsample_bwd_kernel<<<grid_for((long long)C2 * vc.n()), 128, 0, u->stream>>>(gu2, C2, v, u->ge2c);
    relu_bwd_kernel<<<grid_for((long long)C2 * vc.n()), 128, 0, u->stream>>>(u->ge2c, u->a2, (long long)C2 * vc.n());
    conv_bwd_weight(u, 1, u->p1, u->ge2c, vc);
    conv_bwd_data<C1, 27>(u, 1, u->ge2c, vc, u->gp1);
    pool_bwd_add_kernel<<<grid_for((long long)C1 * v.n()), 128, 0, u->stream>>>(u->gp1, C1, v, ge1);
    relu_bwd_kernel<<<grid_for((long long)C1 * v.n()), 128, 0, u->stream>>>(ge1, u->a1, (long long)C1 * v.n());
    conv_bwd_weight(u, 0, x, ge1, v);
    if (cudaGetLastError() != cudaSuccess) return ufail(u, HT_ECUDA, "backward launch failed");
    if (loss) {
        std::vector<float> h(G);
        if (cudaMemcpyAsync(h.data(), u->lpart, G * sizeof(float), cudaMemcpyDeviceToHost, u->stream) != cudaSuccess ||
            cudaStreamSynchronize(u->stream) != cudaSuccess)
            return ufail(u, HT_ECUDA, "loss readback failed");
        double s = 0;
        for (float f : h) s += f;
        *loss = s / (double)ny;
    }
    return HT_OK;
}

bool even_dims(int D, int H, int W) { return D > 1 && H > 1 && W > 1 && D % 2 == 0 && H % 2 == 0 && W % 2 == 0; }

}  // namespace

cudaStream_t ht_unet_stream_internal(ht_unet* u) { return u ? u->stream : nullptr; }

extern "C" {

int ht_unet_create(ht_unet** out, int cin, int cout, int device, void* stream) {
    if (!out || cin < 1 || cin > 16 || cout != 2) return HT_EINVAL;
    ht_unet* u = new ht_unet();
    u->cin = cin;
    u->cout = cout;
    u->device = device;
    cudaSetDevice(device);
    if (stream) u->stream = (cudaStream_t)stream;
    else { cudaStreamCreateWithFlags(&u->stream, cudaStreamNonBlocking); u->own_stream = true; }
    int o = 0;
    for (int l = 0; l < 4; ++l) {
        u->off[l][0] = o;
        o += layer_co(u, l) * layer_ci(u, l) * layer_k(l);
        u->off[l][1] = o;
        o += layer_co(u, l);
    }
    u->np = o;
    if (cudaMalloc(&u->theta, o * sizeof(float)) != cudaSuccess || cudaMalloc(&u->m, o * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&u->v, o * sizeof(float)) != cudaSuccess || cudaMalloc(&u->grad, o * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&u->wb, o * sizeof(__nv_bfloat16)) != cudaSuccess ||
        cudaMalloc(&u->lpart, 1024 * sizeof(float)) != cudaSuccess) {
        ht_unet_destroy(u);
        return HT_ENOMEM;
    }
    cudaMemsetAsync(u->theta, 0, o * sizeof(float), u->stream);
    cudaMemsetAsync(u->m, 0, o * sizeof(float), u->stream);
    cudaMemsetAsync(u->v, 0, o * sizeof(float), u->stream);
    cudaMemsetAsync(u->wb, 0, o * sizeof(__nv_bfloat16), u->stream);
    *out = u;
    return HT_OK;
}

void ht_unet_destroy(ht_unet* u) {
    if (!u) return;
    cudaSetDevice(u->device);
    if (u->stream) cudaStreamSynchronize(u->stream);
    float* bufs[] = {u->theta, u->m, u->v, u->grad, u->a1, u->cat, u->p1, u->a2, u->e2, u->a3, u->d1,
                     u->y, u->gy, u->gd1, u->gcat, u->ge2c, u->gp1, u->ga1, u->lpart};
    for (float* b : bufs)
        if (b) cudaFree(b);
    if (u->wb) cudaFree(u->wb);
    if (u->own_stream && u->stream) cudaStreamDestroy(u->stream);
    delete u;
}

int ht_unet_num_params(const ht_unet* u) { return u ? u->np : 0; }

const char* ht_unet_last_error(const ht_unet* u) { return u ? u->err.c_str() : ""; }

int ht_unet_set_params(ht_unet* u, const float* theta) {
    if (!u || !theta) return HT_EINVAL;
    cudaSetDevice(u->device);
    if (cudaMemcpyAsync(u->theta, theta, u->np * sizeof(float), cudaMemcpyHostToDevice, u->stream) != cudaSuccess)
        return ufail(u, HT_ECUDA, "parameter upload failed");
    to_bf16_kernel<<<(u->np + 255) / 256, 256, 0, u->stream>>>(u->theta, u->wb, u->np);
    cudaMemsetAsync(u->m, 0, u->np * sizeof(float), u->stream);
    cudaMemsetAsync(u->v, 0, u->np * sizeof(float), u->stream);
    u->step = 0;
    return cudaStreamSynchronize(u->stream) == cudaSuccess ? HT_OK : ufail(u, HT_ECUDA, "sync failed");
}

int ht_unet_get_params(ht_unet* u, float* theta) {
    if (!u || !theta) return HT_EINVAL;
    cudaSetDevice(u->device);
    if (cudaMemcpyAsync(theta, u->theta, u->np * sizeof(float), cudaMemcpyDeviceToHost, u->stream) != cudaSuccess ||
        cudaStreamSynchronize(u->stream) != cudaSuccess)
        return ufail(u, HT_ECUDA, "parameter readback failed");
    return HT_OK;
}

int ht_unet_forward(ht_unet* u, const float* x, int D, int H, int W, float* y) {
    if (!u || !x || !y) return HT_EINVAL;
    if (!even_dims(D, H, W)) return ufail(u, HT_EINVAL, "grid sizes must be even and > 1");
    cudaSetDevice(u->device);
    const Vol v{D, H, W};
    int rc = ensure(u, v);
    if (rc != HT_OK) return rc;
    rc = forward(u, x, v);
    if (rc != HT_OK) return rc;
    if (cudaMemcpyAsync(y, u->y, (size_t)u->cout * v.n() * sizeof(float), cudaMemcpyDeviceToDevice, u->stream) !=
        cudaSuccess)
        return ufail(u, HT_ECUDA, "output copy failed");
    return HT_OK;
}

int ht_unet_loss_grad(ht_unet* u, const float* x, const float* target, int D, int H, int W, double* loss,
                      float* grad_host) {
    if (!u || !x || !target) return HT_EINVAL;
    if (!even_dims(D, H, W)) return ufail(u, HT_EINVAL, "grid sizes must be even and > 1");
    cudaSetDevice(u->device);
    const Vol v{D, H, W};
    int rc = ensure(u, v);
    if (rc == HT_OK) rc = forward(u, x, v);
    if (rc == HT_OK) rc = backward(u, x, target, v, loss);
    if (rc == HT_OK && grad_host) {
        if (cudaMemcpyAsync(grad_host, u->grad, u->np * sizeof(float), cudaMemcpyDeviceToHost, u->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(u->stream) != cudaSuccess)
            return ufail(u, HT_ECUDA, "gradient readback failed");
    }
    return rc;
}

int ht_unet_train_step(ht_unet* u, const float* x, const float* target, int D, int H, int W, float lr,
                       double* loss) {
    if (!u || !x || !target || !(lr > 0)) return HT_EINVAL;
    int rc = ht_unet_loss_grad(u, x, target, D, H, W, loss, nullptr);
    if (rc != HT_OK) return rc;
    u->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)u->step), c2 = 1.f - powf(b2, (float)u->step);
    adam_kernel<<<(u->np + 255) / 256, 256, 0, u->stream>>>(u->theta, u->m, u->v, u->grad, u->np, lr, b1, b2, c1, c2,
                                                            1e-8f, u->wb);
    return cudaGetLastError() == cudaSuccess ? HT_OK : ufail(u, HT_ECUDA, "adam launch failed");
}

}  // extern "C"
