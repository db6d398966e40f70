// Learned warm start of the per-step Krylov solves: features of the state
// (the last two increments of T and h), the Darcy flux and the heat sources,
// a U-Net prediction of the next increments, and a gate that keeps the
// previous-step initial guess whenever the learned one has the larger
// residual.  The solver itself is unchanged and converges to the same
// tolerance either way.
#include <cuda_runtime.h>
#include <math.h>

#include "ht_internal.cuh"

cudaStream_t ht_unet_stream_internal(ht_unet* net);

namespace ht {
namespace {

#define LOOP(i, n) \
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

__device__ __forceinline__ double lbsum(double v) {
    __shared__ double ws[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) ws[wid] = v;
    __syncthreads();
    v = (threadIdx.x < (blockDim.x >> 5)) ? ws[lane] : 0.0;
    if (wid == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

// Darcy velocity at node id from the head by differences of neighbouring
// nodes (one-sided on the faces) and the conductivity of the cell whose low
// corner the node is (the last cell along an axis on the high faces): a
// feature of the network, not part of the method's arithmetic
__device__ __forceinline__ void node_flux(const Grid& g, const double* __restrict__ h, const double* __restrict__ K,
                                          double ihx, double ihy, double ihz, long long id, double q[3]) {
    const int i = (int)(id % g.Nx), j = (int)((id / g.Nx) % g.Ny), k = (int)(id / ((long long)g.Nx * g.Ny));
    const int ci = min(i / g.P, g.ncx - 1), cj = min(j / g.P, g.ncy - 1), ck = min(k / g.P, g.ncz - 1);
    const double Kc = K[ci + (long long)g.ncx * (cj + (long long)g.ncy * ck)];
    const long long sx = 1, sy = g.Nx, sz = (long long)g.Nx * g.Ny;
    const int ia = i > 0 ? i - 1 : i, ib = i < g.Nx - 1 ? i + 1 : i;
    const int ja = j > 0 ? j - 1 : j, jb = j < g.Ny - 1 ? j + 1 : j;
    const int ka = k > 0 ? k - 1 : k, kb = k < g.Nz - 1 ? k + 1 : k;
    q[0] = -Kc * (h[id + (ib - i) * sx] - h[id + (ia - i) * sx]) * ihx / (double)max(ib - ia, 1);
    q[1] = -Kc * (h[id + (jb - j) * sy] - h[id + (ja - j) * sy]) * ihy / (double)max(jb - ja, 1);
    q[2] = -Kc * (h[id + (kb - k) * sz] - h[id + (ka - k) * sz]) * ihz / (double)max(kb - ka, 1);
}

// partial sums of dT1^2, dh1^2, |q|^2 and F_T^2
__global__ void sumsq_kernel(const Grid g, const double* __restrict__ a, const double* __restrict__ b,
                             const double* __restrict__ h, const double* __restrict__ K, const double* __restrict__ F,
                             double ihx, double ihy, double ihz, double* __restrict__ part, int stride) {
    double sa = 0, sb = 0, sq = 0, sf = 0;
    LOOP(i, g.nn) {
        sa = fma(a[i], a[i], sa);
        sb = fma(b[i], b[i], sb);
        double q[3];
        node_flux(g, h, K, ihx, ihy, ihz, i, q);
        sq = fma(q[0], q[0], fma(q[1], q[1], fma(q[2], q[2], sq)));
        sf = fma(F[i], F[i], sf);
    }
    sa = lbsum(sa);
    sb = lbsum(sb);
    sq = lbsum(sq);
    sf = lbsum(sf);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = sa;
        part[stride + blockIdx.x] = sb;
        part[2 * (size_t)stride + blockIdx.x] = sq;
        part[3 * (size_t)stride + blockIdx.x] = sf;
    }
}

// padded voxel p -> node id, or -1 in the padding
__device__ __forceinline__ int voxel_node(const Grid& g, int Hp, int Wp, long long p) {
    const int x = (int)(p % Wp), y = (int)((p / Wp) % Hp), z = (int)(p / ((long long)Wp * Hp));
    if (x >= g.Nx || y >= g.Ny || z >= g.Nz) return -1;
    return x + g.Nx * (y + g.Ny * z);
}

// the kLearnFeatures channels [dT1, dT2, dh1, dh2, F_T, q_x, q_y, q_z], each
// divided by its scale (RMS over the nodes; the increments of a field share one)
__global__ void feat_kernel(const Grid g, int Hp, int Wp, long long nv, const double* __restrict__ dT1,
                            const double* __restrict__ dT2, const double* __restrict__ dh1,
                            const double* __restrict__ dh2, const double* __restrict__ h,
                            const double* __restrict__ K, const double* __restrict__ F, double ihx, double ihy,
                            double ihz, double iT, double ih, double iq, double iF, float* __restrict__ f) {
    LOOP(p, nv) {
        const int id = voxel_node(g, Hp, Wp, p);
        float v[kLearnFeatures] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (id >= 0) {
            v[0] = (float)(dT1[id] * iT);
            v[1] = (float)(dT2[id] * iT);
            v[2] = (float)(dh1[id] * ih);
            v[3] = (float)(dh2[id] * ih);
            v[4] = (float)(F[id] * iF);
            double q[3];
            node_flux(g, h, K, ihx, ihy, ihz, id, q);
            v[5] = (float)(q[0] * iq);
            v[6] = (float)(q[1] * iq);
            v[7] = (float)(q[2] * iq);
        }
#pragma unroll
        for (int k = 0; k < kLearnFeatures; ++k) f[k * nv + p] = v[k];
    }
}

// x += s * pred[voxel(id)] on every node
__global__ void guess_kernel(const Grid g, int Hp, int Wp, const float* __restrict__ pred, double s,
                             double* __restrict__ x) {
    LOOP(id, g.nn) {
        const int i = (int)(id % g.Nx), j = (int)((id / g.Nx) % g.Ny), k = (int)(id / ((long long)g.Nx * g.Ny));
        const long long p = (long long)i + (long long)Wp * (j + (long long)Hp * k);
        x[id] += s * (double)pred[p];
    }
}

// new increments: history shift, optional training targets
__global__ void history_kernel(const Grid g, int Hp, int Wp, long long nv, const double* __restrict__ T,
                               const double* __restrict__ Tn, const double* __restrict__ h,
                               const double* __restrict__ hn, double* __restrict__ dT1, double* __restrict__ dT2,
                               double* __restrict__ dh1, double* __restrict__ dh2, double iT, double ih,
                               float* __restrict__ targ) {
    LOOP(id, g.nn) {
        const double tT = T[id] - Tn[id], th = h[id] - hn[id];
        dT2[id] = dT1[id];
        dT1[id] = tT;
        dh2[id] = dh1[id];
        dh1[id] = th;
        if (targ) {
            const int i = (int)(id % g.Nx), j = (int)((id / g.Nx) % g.Ny), k = (int)(id / ((long long)g.Nx * g.Ny));
            const long long p = (long long)i + (long long)Wp * (j + (long long)Hp * k);
            targ[p] = (float)(tT * iT);
            targ[nv + p] = (float)(th * ih);
        }
    }
}

template <typename T>
int lalloc(ht_ctx* c, T** p, size_t n) {
    if (*p) return HT_OK;
    if (cudaMalloc(p, n * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, HT_ENOMEM, "learned-guess buffers do not fit");
    }
    HT_CUDA(c, cudaMemsetAsync(*p, 0, n * sizeof(T), c->stream));
    return HT_OK;
}

int ensure_buffers(ht_ctx* c) {
    const size_t nn = (size_t)c->grid.nn;
    // the network pools three times: grid sizes rounded up to multiples of 8
    c->Dp = (c->grid.Nz + 7) / 8 * 8;
    c->Hp = (c->grid.Ny + 7) / 8 * 8;
    c->Wp = (c->grid.Nx + 7) / 8 * 8;
    const size_t nv = (size_t)c->Dp * c->Hp * c->Wp;
    for (double** p : {&c->hn, &c->Tn, &c->dh1, &c->dh2, &c->dT1, &c->dT2}) HT_TRY(lalloc(c, p, nn));
    HT_TRY(lalloc(c, &c->feat, (size_t)kLearnFeatures * nv));
    HT_TRY(lalloc(c, &c->targ, 2 * nv));
    HT_TRY(lalloc(c, &c->pred, 2 * nv));
    return HT_OK;
}

}  // namespace

int learned_begin(ht_ctx* c) {
    c->have_feat = 0;
    if (!c->net && !c->learn_record) return HT_OK;
    HT_TRY(ensure_buffers(c));
    const size_t nn = (size_t)c->grid.nn;
    HT_CUDA(c, cudaMemcpyAsync(c->hn, c->h, nn * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    HT_CUDA(c, cudaMemcpyAsync(c->Tn, c->T, nn * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    if (c->hist < 2) return HT_OK;
    const int G = vec_grid(c);
    const double ihx = c->grid.P / c->H[0], ihy = c->grid.P / c->H[1], ihz = c->grid.P / c->H[2];
    sumsq_kernel<<<G, kVecThreads, 0, c->stream>>>(c->grid, c->dT1, c->dh1, c->h, c->K64, c->F[HT_TEMP], ihx, ihy,
                                                   ihz, c->part, c->part_stride); ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    std::vector<double> h(4 * (size_t)c->part_stride);
    HT_CUDA(c, cudaMemcpyAsync(h.data(), c->part, 4 * (size_t)c->part_stride * sizeof(double),
                               cudaMemcpyDeviceToHost, c->stream));
    HT_CUDA(c, cudaStreamSynchronize(c->stream));
    double a = 0, b = 0, q = 0, fs = 0;
    for (int i = 0; i < G; ++i) {
        a += h[i];
        b += h[(size_t)c->part_stride + i];
        q += h[2 * (size_t)c->part_stride + i];
        fs += h[3 * (size_t)c->part_stride + i];
    }
    c->lscale_T = a > 0 ? sqrt(a / (double)nn) : 1.0;
    c->lscale_h = b > 0 ? sqrt(b / (double)nn) : 1.0;
    const double sq = q > 0 ? sqrt(q / (double)nn) : 1.0, sF = fs > 0 ? sqrt(fs / (double)nn) : 1.0;
    const long long nv = (long long)c->Dp * c->Hp * c->Wp;
    feat_kernel<<<G, kVecThreads, 0, c->stream>>>(c->grid, c->Hp, c->Wp, nv, c->dT1, c->dT2, c->dh1, c->dh2, c->h,
                                                  c->K64, c->F[HT_TEMP], ihx, ihy, ihz, 1.0 / c->lscale_T,
                                                  1.0 / c->lscale_h, 1.0 / sq, 1.0 / sF, c->feat); ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    c->have_feat = 1;
    if (c->net) {
        // order the network's stream after the features and the solver after the prediction
        cudaStream_t ns = ht_unet_stream_internal(c->net);
        cudaEvent_t e1, e2;
        HT_CUDA(c, cudaEventCreateWithFlags(&e1, cudaEventDisableTiming));
        HT_CUDA(c, cudaEventCreateWithFlags(&e2, cudaEventDisableTiming));
        HT_CUDA(c, cudaEventRecord(e1, c->stream));
        HT_CUDA(c, cudaStreamWaitEvent(ns, e1, 0));
        const int rc = ht_unet_forward(c->net, c->feat, c->Dp, c->Hp, c->Wp, c->pred);
        HT_CUDA(c, cudaEventRecord(e2, ns));
        HT_CUDA(c, cudaStreamWaitEvent(c->stream, e2, 0));
        cudaEventDestroy(e1);
        cudaEventDestroy(e2);
        if (rc != HT_OK) return fail(c, rc, "U-Net forward failed: %s", ht_unet_last_error(c->net));
    }
    return HT_OK;
}

int learned_gate(ht_ctx* c, int field, double dt, double* x, const double* b, int* used, double* res) {
    *used = 0;
    *res = -1.0;
    if (!c->net || !c->have_feat) return HT_OK;
    // the gate compares the two guesses by the residual with the FP32
    // operator (FP64 right-hand side): enough to rank them, and a fraction of
    // the cost of an FP64 apply
    double r0 = 0, rL = 0;
    HT_TRY(fast_residual(c, field, dt, x, b, &r0));
    const size_t nn = (size_t)c->grid.nn;
    HT_CUDA(c, cudaMemcpyAsync(c->z, x, nn * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    const long long nv = (long long)c->Dp * c->Hp * c->Wp;
    const float* pr = c->pred + (field == HT_TEMP ? 0 : nv);
    const double s = field == HT_TEMP ? c->lscale_T : c->lscale_h;
    guess_kernel<<<vec_grid(c), kVecThreads, 0, c->stream>>>(c->grid, c->Hp, c->Wp, pr, s, c->z); ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    HT_TRY(set_dirichlet_values(c, field, c->z));
    HT_TRY(fast_residual(c, field, dt, c->z, b, &rL));
    if (rL < r0) {
        HT_CUDA(c, cudaMemcpyAsync(x, c->z, nn * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
        *used = 1;
        *res = rL;
    } else {
        *res = r0;
    }
    return HT_OK;
}

int learned_end(ht_ctx* c) {
    if (!c->net && !c->learn_record) return HT_OK;
    if (!c->hn) return HT_OK;
    const long long nv = (long long)c->Dp * c->Hp * c->Wp;
    float* targ = (c->learn_record && c->have_feat) ? c->targ : nullptr;
    history_kernel<<<vec_grid(c), kVecThreads, 0, c->stream>>>(c->grid, c->Hp, c->Wp, nv, c->T, c->Tn, c->h, c->hn,
                                                               c->dT1, c->dT2, c->dh1, c->dh2, 1.0 / c->lscale_T,
                                                               1.0 / c->lscale_h, targ); ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    c->have_sample = targ ? 1 : 0;
    if (c->hist < 2) c->hist += 1;
    return HT_OK;
}

void learned_free(ht_ctx* c) {
    for (double* p : {c->hn, c->Tn, c->dh1, c->dh2, c->dT1, c->dT2})
        if (p) cudaFree(p);
    for (float* p : {c->feat, c->targ, c->pred})
        if (p) cudaFree(p);
    c->hn = c->Tn = c->dh1 = c->dh2 = c->dT1 = c->dT2 = nullptr;
    c->feat = c->targ = c->pred = nullptr;
}

}  // namespace ht

using namespace ht;

extern "C" {

int ht_set_learned_guess(ht_ctx* c, ht_unet* net, int record) {
    if (!c) return HT_EINVAL;
    c->net = net;
    c->learn_record = record ? 1 : 0;
    return HT_OK;
}

int ht_learned_sample(ht_ctx* c, float* features, float* targets, int* dims) {
    if (!c || !features || !targets || !dims) return HT_EINVAL;
    if (!c->have_sample) return fail(c, HT_EINVAL, "no complete learned-guess sample yet");
    cudaSetDevice(c->device);
    const size_t nv = (size_t)c->Dp * c->Hp * c->Wp;
    HT_CUDA(c, cudaMemcpyAsync(features, c->feat, (size_t)kLearnFeatures * nv * sizeof(float), cudaMemcpyDeviceToDevice,
                               c->stream));
    HT_CUDA(c, cudaMemcpyAsync(targets, c->targ, 2 * nv * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
    HT_CUDA(c, cudaStreamSynchronize(c->stream));
    dims[0] = c->Dp;
    dims[1] = c->Hp;
    dims[2] = c->Wp;
    return HT_OK;
}

}  // extern "C"
