// Batched time steps of many independent problems (same element order, any
// mesh sizes): the inner FP32 head CG of all problems runs as one launch per
// phase over a work list of (problem, block) items, and a chunk of CG
// iterations is captured once in a CUDA graph and replayed until every
// problem has converged.  Everything else (loads, right-hand sides, FP64
// defect-correction residuals, heat solves) uses the single-problem path.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "ht_internal.cuh"

#include <atomic>
#include <functional>
#include <string>
#include <thread>

namespace ht {

namespace {

// per-problem descriptor, device resident
struct BProb {
    Grid g;
    float Ss, dt;
    const float* K;
    float *x, *r, *p, *q, *Dinv, *E;
    double* part;
    int stride;
    Scal* sc;
    int cell_gx, cell_gy, cell_zs, zlen;
    int node_nx, node_ny, node_ks, klen;
    int vec_blocks;
    int cell_item0, node_item0, vec_item0;
    Elem<float> e;
};

__device__ __forceinline__ bool b_on_dir(const Grid& g, int i, int j, int k) {
    const int m = g.dmask;
    return ((m & 1) && i == 0) || ((m & 2) && i == g.Nx - 1) || ((m & 4) && j == 0) ||
           ((m & 8) && j == g.Ny - 1) || ((m & 16) && k == 0) || ((m & 32) && k == g.Nz - 1);
}

__device__ __forceinline__ double b_block_sum(double v) {
    __shared__ double ws[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int lane = tid & 31, wid = tid >> 5;
    __syncthreads();
    if (lane == 0) ws[wid] = v;
    __syncthreads();
    const int nw = (blockDim.x * blockDim.y + 31) >> 5;
    v = (tid < nw) ? ws[lane] : 0.0;
    if (wid == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

__device__ double b_reduce(const double* part, int np) {
    double s = 0.0;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int nt = blockDim.x * blockDim.y;
    for (int i = tid; i < np; i += nt) s += part[i];
    return b_block_sum(s);
}

template <int n, int AX, bool TR>
__device__ __forceinline__ void b_sweep(float (&u)[n * n * n], const float (&M)[3][3]) {
    constexpr int st = AX == 0 ? 1 : (AX == 1 ? n : n * n);
#pragma unroll
    for (int l = 0; l < n * n; ++l) {
        int base;
        if (AX == 0) base = l * n;
        else if (AX == 1) base = (l % n) + (l / n) * n * n;
        else base = l;
        float in[n], out[n];
#pragma unroll
        for (int a = 0; a < n; ++a) in[a] = u[base + a * st];
#pragma unroll
        for (int i = 0; i < n; ++i) {
            float s = 0.f;
#pragma unroll
            for (int a = 0; a < n; ++a) s = fmaf(TR ? M[a][i] : M[i][a], in[a], s);
            out[i] = s;
        }
#pragma unroll
        for (int i = 0; i < n; ++i) u[base + i * st] = out[i];
    }
}

// cell pass of the head apply (fast diagonalisation) for all problems
template <int P>
__global__ void __launch_bounds__(128) bcell_kernel(const BProb* __restrict__ probs,
                                                    const int* __restrict__ item_prob) {
    constexpr int n = P + 1, NL = n * n * n;
    __shared__ BProb pr;
    const int pi = item_prob[blockIdx.x];
    if (threadIdx.x == 0 && threadIdx.y == 0) pr = probs[pi];
    __syncthreads();
    if (pr.sc->done) return;
    const Grid& g = pr.g;
    const int local = blockIdx.x - pr.cell_item0;
    const int bx = local % pr.cell_gx, t = local / pr.cell_gx, by = t % pr.cell_gy, bz = t / pr.cell_gy;
    const int cx = bx * 32 + threadIdx.x, cy = by * 4 + threadIdx.y;
    if (cx >= g.ncx || cy >= g.ncy) return;
    const int cz0 = bz * pr.zlen, cz1 = min(cz0 + pr.zlen, g.ncz);
    const int nc = (int)g.nc, layer = g.ncx * g.ncy;
    const int NX = g.Nx, NXY = g.Nx * g.Ny;
    const bool edge_xy = g.dmask != 0 && (cx == 0 || cx == g.ncx - 1 || cy == 0 || cy == g.ncy - 1);
    const float* x = pr.p;
    int base = P * cx + NX * P * cy + NXY * P * cz0;
    int c = cx + g.ncx * cy + layer * cz0;
    for (int cz = cz0; cz < cz1; ++cz, base += NXY * P, c += layer) {
        float u[NL];
#pragma unroll
        for (int c2 = 0; c2 < n; ++c2)
#pragma unroll
            for (int b = 0; b < n; ++b)
#pragma unroll
                for (int a = 0; a < n; ++a) u[a + n * (b + n * c2)] = __ldg(x + base + NX * b + NXY * c2 + a);
        if (edge_xy || (g.dmask & 48 && (cz == 0 || cz == g.ncz - 1))) {
#pragma unroll
            for (int c2 = 0; c2 < n; ++c2)
#pragma unroll
                for (int b = 0; b < n; ++b)
#pragma unroll
                    for (int a = 0; a < n; ++a)
                        if (b_on_dir(g, P * cx + a, P * cy + b, P * cz + c2)) u[a + n * (b + n * c2)] = 0.f;
        }
        const float beta = pr.dt * __ldg(pr.K + c);
        b_sweep<n, 0, false>(u, pr.e.G[0]);
        b_sweep<n, 1, false>(u, pr.e.G[1]);
        b_sweep<n, 2, false>(u, pr.e.G[2]);
#pragma unroll
        for (int l = 0; l < NL; ++l) u[l] *= fmaf(beta, pr.e.LS[l], pr.Ss);
        b_sweep<n, 2, true>(u, pr.e.G[2]);
        b_sweep<n, 1, true>(u, pr.e.G[1]);
        b_sweep<n, 0, true>(u, pr.e.G[0]);
#pragma unroll
        for (int l = 0; l < NL; ++l) pr.E[l * nc + c] = u[l];
    }
}

// node pass: q = sum of cell contributions, p.q partials per problem
template <int P>
__global__ void __launch_bounds__(128) bnode_kernel(const BProb* __restrict__ probs,
                                                    const int* __restrict__ item_prob) {
    constexpr int n = P + 1;
    __shared__ BProb pr;
    const int pi = item_prob[blockIdx.x];
    if (threadIdx.x == 0 && threadIdx.y == 0) pr = probs[pi];
    __syncthreads();
    if (pr.sc->done) return;
    const Grid& g = pr.g;
    const int local = blockIdx.x - pr.node_item0;
    const int bx = local % pr.node_nx, t = local / pr.node_nx, by = t % pr.node_ny, bz = t / pr.node_ny;
    const int i = bx * 32 + threadIdx.x, j = by * 4 + threadIdx.y;
    float dot = 0.f;
    if (i < g.Nx && j < g.Ny) {
        const int nc = (int)g.nc, layer = g.ncx * g.ncy;
        int cxy[4], lxy[4];
        bool vxy[4];
        {
            int cxs[2] = {0, 0}, axs[2] = {0, 0}, cys[2] = {0, 0}, bys[2] = {0, 0};
            bool vx[2] = {false, false}, vy[2] = {false, false};
            if (i % P == 0) {
                if (i / P - 1 >= 0) { cxs[0] = i / P - 1; axs[0] = P; vx[0] = true; }
                if (i / P < g.ncx) { cxs[1] = i / P; axs[1] = 0; vx[1] = true; }
            } else { cxs[0] = i / P; axs[0] = i % P; vx[0] = true; }
            if (j % P == 0) {
                if (j / P - 1 >= 0) { cys[0] = j / P - 1; bys[0] = P; vy[0] = true; }
                if (j / P < g.ncy) { cys[1] = j / P; bys[1] = 0; vy[1] = true; }
            } else { cys[0] = j / P; bys[0] = j % P; vy[0] = true; }
#pragma unroll
            for (int yy = 0; yy < 2; ++yy)
#pragma unroll
                for (int xx = 0; xx < 2; ++xx) {
                    const int q = xx + 2 * yy;
                    vxy[q] = vx[xx] && vy[yy];
                    cxy[q] = cxs[xx] + g.ncx * cys[yy];
                    lxy[q] = axs[xx] + n * bys[yy];
                }
        }
        const bool dir_xy = ((g.dmask & 1) && i == 0) || ((g.dmask & 2) && i == g.Nx - 1) ||
                            ((g.dmask & 4) && j == 0) || ((g.dmask & 8) && j == g.Ny - 1);
        const int k0 = bz * pr.klen, k1 = min(k0 + pr.klen, g.Nz);
        const int NXY = g.Nx * g.Ny;
        int id = i + g.Nx * j + NXY * k0;
        for (int k = k0; k < k1; ++k, id += NXY) {
            int czs[2] = {0, 0}, czl[2] = {0, 0};
            bool vz[2] = {false, false};
            if (k % P == 0) {
                if (k / P - 1 >= 0) { czs[0] = k / P - 1; czl[0] = P; vz[0] = true; }
                if (k / P < g.ncz) { czs[1] = k / P; czl[1] = 0; vz[1] = true; }
            } else { czs[0] = k / P; czl[0] = k % P; vz[0] = true; }
            float v[8];
#pragma unroll
            for (int zz = 0; zz < 2; ++zz) {
                const int cz = layer * czs[zz], lz = n * n * czl[zz];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    v[q + 4 * zz] = (vz[zz] && vxy[q]) ? __ldg(pr.E + (lxy[q] + lz) * nc + cxy[q] + cz) : 0.f;
            }
            const float sum = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
            const float xv = pr.p[id];
            const bool d = dir_xy || ((g.dmask & 16) && k == 0) || ((g.dmask & 32) && k == g.Nz - 1);
            const float yv = d ? xv : sum;
            pr.q[id] = yv;
            dot = fmaf(xv, yv, dot);
        }
    }
    const double tot = b_block_sum((double)dot);
    if (threadIdx.x == 0 && threadIdx.y == 0) pr.part[local] = tot;
}

// x += alpha p; r -= alpha q; partials r.z, r.r (slots 1, 2)
__global__ void __launch_bounds__(256) bupdate_kernel(const BProb* __restrict__ probs,
                                                      const int* __restrict__ item_prob, int par) {
    __shared__ double sh;
    const int pi = item_prob[blockIdx.x];
    const BProb& pr = probs[pi];
    Scal* s = pr.sc;
    if (s->done) return;
    const int np = pr.node_nx * pr.node_ny * pr.node_ks;
    const double pq = b_reduce(pr.part, np);
    if (threadIdx.x == 0) sh = pq;
    __syncthreads();
    const int local = blockIdx.x - pr.vec_item0;
    if (!(sh > 0.0) || !isfinite(sh)) {
        if (local == 0 && threadIdx.x == 0) { s->status = ST_BREAKDOWN; s->done = 1; }
        return;
    }
    const float alpha = (float)(s->rz2[par] / sh);
    const int nn = (int)pr.g.nn;
    float rz = 0.f, rr = 0.f;
    for (int i = local * blockDim.x + threadIdx.x; i < nn; i += pr.vec_blocks * blockDim.x) {
        pr.x[i] = fmaf(alpha, pr.p[i], pr.x[i]);
        const float ri = fmaf(-alpha, pr.q[i], pr.r[i]);
        pr.r[i] = ri;
        rz = fmaf(ri, pr.Dinv[i] * ri, rz);
        rr = fmaf(ri, ri, rr);
    }
    const double a = b_block_sum((double)rz);
    const double b = b_block_sum((double)rr);
    if (threadIdx.x == 0) {
        pr.part[(size_t)pr.stride + local] = a;
        pr.part[(size_t)2 * pr.stride + local] = b;
    }
}

// p = Dinv r + beta p; the problem's first item stores the new scalars
__global__ void __launch_bounds__(256) bpupdate_kernel(const BProb* __restrict__ probs,
                                                       const int* __restrict__ item_prob, int par, double tol2,
                                                       int max_iter) {
    __shared__ double sh[2];
    const int pi = item_prob[blockIdx.x];
    const BProb& pr = probs[pi];
    Scal* s = pr.sc;
    if (s->done) return;
    const double rz = b_reduce(pr.part + pr.stride, pr.vec_blocks);
    if (threadIdx.x == 0) sh[0] = rz;
    const double rr = b_reduce(pr.part + 2 * (size_t)pr.stride, pr.vec_blocks);
    if (threadIdx.x == 0) sh[1] = rr;
    __syncthreads();
    const int local = blockIdx.x - pr.vec_item0;
    const float beta = (float)(sh[0] / s->rz2[par]);
    if (local == 0 && threadIdx.x == 0) {
        s->rz2[par ^ 1] = sh[0];
        s->rr = sh[1];
        s->iters += 1;
        if (!isfinite(sh[0]) || !isfinite(sh[1])) { s->status = ST_NAN; s->done = 1; }
        else if (sh[1] <= tol2 * s->bb || s->iters >= max_iter) s->done = 1;
    }
    const int nn = (int)pr.g.nn;
    for (int i = local * blockDim.x + threadIdx.x; i < nn; i += pr.vec_blocks * blockDim.x)
        pr.p[i] = fmaf(beta, pr.p[i], pr.Dinv[i] * pr.r[i]);
}

// done flags of all problems into one array (one copy to the host)
__global__ void bcollect_kernel(const BProb* __restrict__ probs, int n, int* __restrict__ done) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) done[i] = probs[i].sc->done;
}

}  // namespace
}  // namespace ht

struct ht_batch {
    std::vector<ht_ctx*> probs;
    int device = 0;
    int order = 1;
    cudaStream_t stream = nullptr;
    ht::BProb* d_probs = nullptr;
    int *d_cell_item = nullptr, *d_node_item = nullptr, *d_vec_item = nullptr, *d_done = nullptr;
    int *h_done = nullptr;
    int n_cell = 0, n_node = 0, n_vec = 0;
    cudaGraphExec_t graph = nullptr;
    double graph_dt = -1.0;
    int mode = HT_BATCH_CONCURRENT;
    std::string err;
    // persistent mode
    ht::Q1Batch q1;
    int planes = 0;            // node planes per z chunk (0: automatic)
    double wait_ms = 2000.0;   // bound of each grid-barrier wait
    int drop_cta = -1;         // failure injection (tests): CTA that skips its first arrival
    int last_err_cta = -1;
};

namespace ht {
namespace {

constexpr int kGraphIters = 4;   // CG iterations per graph replay (even: r.z parity repeats)

int bfail(ht_batch* b, int code, const char* msg) {
    if (b) b->err = msg;
    return code;
}

// build descriptors and work lists for the current dt
int batch_prepare(ht_batch* b, double dt) {
    const int np = (int)b->probs.size();
    std::vector<BProb> h(np);
    std::vector<int> cell_item, node_item, vec_item;
    for (int i = 0; i < np; ++i) {
        ht_ctx* c = b->probs[i];
        BProb& pr = h[i];
        memset(&pr, 0, sizeof(pr));
        pr.g = c->grid;
        pr.g.dmask = c->dmask[HT_HEAD];
        pr.Ss = (float)c->Ss;
        pr.dt = (float)dt;
        pr.K = c->K32;
        pr.x = c->d32; pr.r = c->r32; pr.p = c->p32; pr.q = c->q32; pr.Dinv = c->D32; pr.E = c->E32 + kElemPad;
        pr.part = c->part;
        pr.stride = c->part_stride;
        pr.sc = c->scal + 1;
        pr.e = c->e32;
        const Grid& g = pr.g;
        pr.cell_gx = (g.ncx + 31) / 32;
        pr.cell_gy = (g.ncy + 3) / 4;
        pr.cell_zs = g.ncz;
        pr.zlen = 1;
        pr.node_nx = (g.Nx + 31) / 32;
        pr.node_ny = (g.Ny + 3) / 4;
        int ks = g.Nz;
        const int kmax = c->part_stride / (pr.node_nx * pr.node_ny);
        if (ks > kmax) ks = kmax > 0 ? kmax : 1;
        pr.klen = (g.Nz + ks - 1) / ks;
        pr.node_ks = (g.Nz + pr.klen - 1) / pr.klen;
        pr.vec_blocks = (int)std::min<long long>((g.nn + 255) / 256, 64);
        pr.cell_item0 = (int)cell_item.size();
        for (int k = 0; k < pr.cell_gx * pr.cell_gy * pr.cell_zs; ++k) cell_item.push_back(i);
        pr.node_item0 = (int)node_item.size();
        for (int k = 0; k < pr.node_nx * pr.node_ny * pr.node_ks; ++k) node_item.push_back(i);
        pr.vec_item0 = (int)vec_item.size();
        for (int k = 0; k < pr.vec_blocks; ++k) vec_item.push_back(i);
    }
    auto upload = [&](int** dst, const std::vector<int>& v) -> int {
        if (*dst) cudaFree(*dst);
        *dst = nullptr;
        if (cudaMalloc(dst, v.size() * sizeof(int)) != cudaSuccess) return HT_ENOMEM;
        return cudaMemcpyAsync(*dst, v.data(), v.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream) ==
                       cudaSuccess ? HT_OK : HT_ECUDA;
    };
    int rc = upload(&b->d_cell_item, cell_item);
    if (rc == HT_OK) rc = upload(&b->d_node_item, node_item);
    if (rc == HT_OK) rc = upload(&b->d_vec_item, vec_item);
    if (rc != HT_OK) return bfail(b, rc, "work-list upload failed");
    b->n_cell = (int)cell_item.size();
    b->n_node = (int)node_item.size();
    b->n_vec = (int)vec_item.size();
    if (cudaMemcpyAsync(b->d_probs, h.data(), np * sizeof(BProb), cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
        return bfail(b, HT_ECUDA, "descriptor upload failed");
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return bfail(b, HT_ECUDA, "sync failed");
    return HT_OK;
}

int enqueue_iterations(ht_batch* b, double tol, int max_iter) {
    const int np = (int)b->probs.size();
    for (int it = 0; it < kGraphIters; ++it) {
        const int par = it & 1;
        if (b->order == 1) {
            bcell_kernel<1><<<b->n_cell, dim3(32, 4), 0, b->stream>>>(b->d_probs, b->d_cell_item);
            bnode_kernel<1><<<b->n_node, dim3(32, 4), 0, b->stream>>>(b->d_probs, b->d_node_item);
        } else {
            bcell_kernel<2><<<b->n_cell, dim3(32, 4), 0, b->stream>>>(b->d_probs, b->d_cell_item);
            bnode_kernel<2><<<b->n_node, dim3(32, 4), 0, b->stream>>>(b->d_probs, b->d_node_item);
        }
        bupdate_kernel<<<b->n_vec, 256, 0, b->stream>>>(b->d_probs, b->d_vec_item, par);
        bpupdate_kernel<<<b->n_vec, 256, 0, b->stream>>>(b->d_probs, b->d_vec_item, par, tol * tol, max_iter);
    }
    bcollect_kernel<<<(np + 127) / 128, 128, 0, b->stream>>>(b->d_probs, np, b->d_done);
    return cudaGetLastError() == cudaSuccess ? HT_OK : HT_ECUDA;
}

// batched inner FP32 CG on A32 d = r32 for the listed problems (slot-1
// scalars already initialised by the per-problem init)
int batch_inner_cg(ht_batch* b, double dt, double tol, int max_iter) {
    const int np = (int)b->probs.size();
    if (!b->graph || b->graph_dt != dt) {
        if (b->graph) cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        int rc = batch_prepare(b, dt);
        if (rc != HT_OK) return rc;
        cudaGraph_t graph;
        if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return bfail(b, HT_ECUDA, "stream capture failed");
        rc = enqueue_iterations(b, tol, max_iter);
        if (cudaStreamEndCapture(b->stream, &graph) != cudaSuccess || rc != HT_OK)
            return bfail(b, HT_ECUDA, "stream capture failed");
        if (cudaGraphInstantiate(&b->graph, graph, 0) != cudaSuccess) {
            cudaGraphDestroy(graph);
            return bfail(b, HT_ECUDA, "graph instantiation failed");
        }
        cudaGraphDestroy(graph);
        b->graph_dt = dt;
    }
    for (int rep = 0; rep * kGraphIters < max_iter; ++rep) {
        if (cudaGraphLaunch(b->graph, b->stream) != cudaSuccess) return bfail(b, HT_ECUDA, "graph launch failed");
        for (ht_ctx* c : b->probs) c->n_launch += 4 * kGraphIters + 1;
        if (cudaMemcpyAsync(b->h_done, b->d_done, np * sizeof(int), cudaMemcpyDeviceToHost, b->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(b->stream) != cudaSuccess)
            return bfail(b, HT_ECUDA, "done-flag readback failed");
        bool all = true;
        for (int i = 0; i < np; ++i) all = all && b->h_done[i];
        if (all) return HT_OK;
    }
    return HT_OK;
}

}  // namespace

// pieces of the single-problem path used by the batch (ht_krylov.cu / ht_capi.cu)
int batch_head_begin(ht_ctx* c, double dt);
int batch_outer_residual(ht_ctx* c, double dt, double tol, int* converged, double* res);
int batch_inner_init(ht_ctx* c, double dt, double inner_tol, int max_iter);
int batch_outer_update(ht_ctx* c);
int batch_outer_residual_enqueue(ht_ctx* c, double dt);
int batch_outer_residual_read(ht_ctx* c, double tol, int* converged, double* res);
int batch_outer_update_enqueue(ht_ctx* c);
int batch_head_end_and_heat(ht_ctx* c, double dt, ht_step_stats* st);

}  // namespace ht

using namespace ht;

extern "C" {

int ht_batch_create(ht_batch** out, int n, ht_ctx* const* problems) {
    if (!out || n < 1 || !problems) return HT_EINVAL;
    *out = nullptr;
    ht_batch* b = new ht_batch();
    b->device = problems[0]->device;
    b->order = problems[0]->grid.P;
    for (int i = 0; i < n; ++i) {
        ht_ctx* c = problems[i];
        if (!c || c->device != b->device || c->grid.P != b->order) {
            delete b;
            return HT_EINVAL;
        }
        b->probs.push_back(c);
    }
    cudaSetDevice(b->device);
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc(&b->d_probs, n * sizeof(BProb)) != cudaSuccess ||
        cudaMalloc(&b->d_done, n * sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&b->h_done, n * sizeof(int)) != cudaSuccess) {
        ht_batch_destroy(b);
        return HT_ENOMEM;
    }
    *out = b;
    return HT_OK;
}

void ht_batch_destroy(ht_batch* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    q1_batch_free(b->q1);
    for (int* p : {b->d_cell_item, b->d_node_item, b->d_vec_item, b->d_done})
        if (p) cudaFree(p);
    if (b->d_probs) cudaFree(b->d_probs);
    if (b->h_done) cudaFreeHost(b->h_done);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

const char* ht_batch_last_error(const ht_batch* b) { return b ? b->err.c_str() : ""; }

int ht_batch_set_mode(ht_batch* b, int mode) {
    if (!b) return HT_EINVAL;
    if (mode != HT_BATCH_CONCURRENT && mode != HT_BATCH_SHARED_LAUNCHES && mode != HT_BATCH_PERSISTENT)
        return bfail(b, HT_EINVAL, "unknown mode");
    if (mode == HT_BATCH_PERSISTENT)
        for (const ht_ctx* c : b->probs)
            if (!q1_cg_available(c, 1))
                return bfail(b, HT_EINVAL, "the persistent mode needs Q1 problems that use the single-pass kernels");
    b->mode = mode;
    return HT_OK;
}

int ht_batch_set_persistent(ht_batch* b, int planes, double wait_ms, int drop_cta) {
    if (!b) return HT_EINVAL;
    if (planes < 0 || !(wait_ms > 0.0) || !(wait_ms <= 6.0e4) || drop_cta < -1)
        return bfail(b, HT_EINVAL, "planes >= 0, 0 < wait_ms <= 60000 and drop_cta >= -1 are required");
    b->planes = planes;
    b->wait_ms = wait_ms;
    b->drop_cta = drop_cta;
    return HT_OK;
}

int ht_batch_persistent_info(const ht_batch* b, int* planes, int* items, int* grid, int* err_cta) {
    if (!b) return HT_EINVAL;
    if (planes) *planes = b->q1.planes;
    if (items) *items = b->q1.nitems;
    if (grid) *grid = b->q1.grid;
    if (err_cta) *err_cta = b->last_err_cta;
    return HT_OK;
}

// fn(i) for every problem, on worker threads when the problems have
// streams of their own (one thread otherwise)
static void for_each_problem(ht_batch* b, const std::function<void(int)>& fn) {
    const int np = (int)b->probs.size();
    bool shared = false;
    for (int i = 0; i < np && !shared; ++i)
        for (int j = 0; j < i && !shared; ++j) shared = b->probs[i]->stream == b->probs[j]->stream;
    std::atomic<int> next(0);
    auto work = [&] {
        cudaSetDevice(b->device);
        for (int i = next++; i < np; i = next++) fn(i);
    };
    const int nt = shared ? 1 : std::min(np, 8);
    if (nt <= 1) {
        work();
    } else {
        std::vector<std::thread> pool;
        for (int t = 0; t < nt; ++t) pool.emplace_back(work);
        for (auto& th : pool) th.join();
    }
}

// concurrent mode: worker threads step the problems on their own streams
static int batch_step_concurrent(ht_batch* b, double dt, ht_step_stats* stats) {
    const int np = (int)b->probs.size();
    std::vector<int> rcs(np, HT_OK);
    std::vector<ht_step_stats> st(np);
    for_each_problem(b, [&](int i) { rcs[i] = ht_step(b->probs[i], dt, &st[i]); });
    int rc = HT_OK;
    for (int i = 0; i < np; ++i) {
        if (stats) stats[i] = st[i];
        if (rcs[i] != HT_OK && rc == HT_OK) {
            rc = rcs[i];
            b->err = std::string("problem ") + std::to_string(i) + ": " + ht_last_error(b->probs[i]);
        }
    }
    return rc;
}

// persistent mode: the per-problem set-up and the heat solves run on the
// problems' own streams (worker threads); the head solves of all problems
// run on the batch stream, their inner FP32 CG as one cooperative launch per
// outer pass (q1_cg_batch_kernel), their outer residuals and updates
// enqueued for all problems before a single host wait
static int batch_step_persistent(ht_batch* b, double dt, ht_step_stats* stats) {
    const int np = (int)b->probs.size();
    std::vector<int> rcs(np, HT_OK);
    for_each_problem(b, [&](int i) {
        ht_ctx* c = b->probs[i];
        rcs[i] = batch_head_begin(c, dt);
        if (rcs[i] == HT_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) rcs[i] = HT_ECUDA;
    });
    for (int i = 0; i < np; ++i)
        if (rcs[i] != HT_OK) {
            b->err = std::string("problem ") + std::to_string(i) + ": " + ht_last_error(b->probs[i]);
            return rcs[i];
        }
    std::vector<cudaStream_t> saved(np);
    for (int i = 0; i < np; ++i) {
        saved[i] = b->probs[i]->stream;
        b->probs[i]->stream = b->stream;
    }
    auto restore = [&] {
        cudaStreamSynchronize(b->stream);
        for (int i = 0; i < np; ++i) b->probs[i]->stream = saved[i];
    };
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, b->stream);
    int rc = HT_OK;
    rc = q1_batch_prepare(b->q1, b->probs.data(), np, dt, b->planes, b->stream, &b->err);
    std::vector<int> conv(np, 0), outer(np, 0), inner(np, 0);
    std::vector<double> res(np, 0.0);
    const ht_ctx* c0 = b->probs[0];
    const double tol = c0->opts.tol;
    const int max_outer = c0->opts.max_outer > 0 ? c0->opts.max_outer : 30;
    const double base = c0->opts.inner_tol > 0 ? c0->opts.inner_tol : 1e-4;
    int clock_khz = 0;
    cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, b->device);
    const long long budget = (long long)(b->wait_ms * (clock_khz > 0 ? clock_khz : 2000000));
    b->last_err_cta = -1;
    for (int k = 0; k <= max_outer && rc == HT_OK; ++k) {
        for (int i = 0; i < np && rc == HT_OK; ++i)
            if (!conv[i]) rc = batch_outer_residual_enqueue(b->probs[i], dt);
        if (rc == HT_OK && cudaStreamSynchronize(b->stream) != cudaSuccess) rc = bfail(b, HT_ECUDA, "sync failed");
        bool all = true;
        for (int i = 0; i < np && rc == HT_OK; ++i) {
            if (conv[i]) continue;
            rc = batch_outer_residual_read(b->probs[i], tol, &conv[i], &res[i]);
            if (rc != HT_OK) b->err = b->probs[i]->err;
            outer[i] = k;
            all = all && conv[i];
        }
        if (rc != HT_OK || all) break;
        if (k == max_outer) { rc = bfail(b, HT_ENOCONV, "batched head solve did not converge"); break; }
        for (int i = 0; i < np && rc == HT_OK; ++i) {
            ht_ctx* c = b->probs[i];
            // no inner reduction beyond what the outer tolerance needs; a
            // converged problem gets tolerance 1 and is done at once
            const double need = res[i] > 0 ? 0.5 * tol / res[i] : 1.0;
            const double itol = std::max(base, std::min(need, 0.5));
            rc = batch_inner_init(c, dt, conv[i] ? 1.0 : itol, c->opts.max_iter);
        }
        int running = 0, err_cta = -1;
        if (rc == HT_OK) {
            rc = q1_batch_run(b->q1, b->stream, c0->opts.max_iter, budget, k == 0 ? b->drop_cta : -1, &running,
                              &err_cta, &b->err);
            for (ht_ctx* c : b->probs) c->n_launch += 1;
            b->last_err_cta = err_cta;
        }
        for (int i = 0; i < np && rc == HT_OK; ++i)
            if (!conv[i]) rc = batch_outer_update_enqueue(b->probs[i]);
        if (rc == HT_OK && cudaStreamSynchronize(b->stream) != cudaSuccess) rc = bfail(b, HT_ECUDA, "sync failed");
        for (int i = 0; i < np && rc == HT_OK; ++i) {
            if (conv[i]) continue;
            const Scal& s1 = b->probs[i]->scal_host[1];
            if (s1.status == ST_NAN) rc = bfail(b, HT_EINVAL, "batched head solve: FP32 inner solve produced non-finite values");
            inner[i] += s1.iters;
        }
    }
    cudaEventRecord(e1, b->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    restore();
    std::vector<ht_step_stats> st(np);
    if (rc == HT_OK) {
        for_each_problem(b, [&](int i) { rcs[i] = batch_head_end_and_heat(b->probs[i], dt, &st[i]); });
        for (int i = 0; i < np && rc == HT_OK; ++i)
            if (rcs[i] != HT_OK) {
                rc = rcs[i];
                b->err = std::string("problem ") + std::to_string(i) + ": " + ht_last_error(b->probs[i]);
            }
    }
    if (stats)
        for (int i = 0; i < np; ++i) {
            stats[i] = st[i];
            stats[i].iters_head = inner[i];
            stats[i].outer_head = outer[i];
            stats[i].res_head = res[i];
            stats[i].ms_head = ms;
        }
    return rc;
}

int ht_batch_step(ht_batch* b, double dt, ht_step_stats* stats) {
    if (!b) return HT_EINVAL;
    if (!(dt > 0)) return bfail(b, HT_EINVAL, "dt must be positive");
    cudaSetDevice(b->device);
    const int np = (int)b->probs.size();
    for (int i = 0; i < np; ++i) {
        const ht_ctx* c = b->probs[i];
        if (c->opts.precision != HT_MIXED || c->opts.precond != HT_PREC_JACOBI)
            return bfail(b, HT_EINVAL, "batched problems need precision HT_MIXED with the Jacobi preconditioner");
    }
    if (b->mode == HT_BATCH_CONCURRENT) return batch_step_concurrent(b, dt, stats);
    for (const ht_ctx* c : b->probs)
        if (c->graded)
            return bfail(b, HT_EINVAL, "graded meshes are batched in the concurrent mode only");
    if (b->mode == HT_BATCH_PERSISTENT) return batch_step_persistent(b, dt, stats);
    // every problem works on the batch stream for the duration of the step
    std::vector<cudaStream_t> saved(np);
    for (int i = 0; i < np; ++i) {
        ht_ctx* c = b->probs[i];
        cudaStreamSynchronize(c->stream);
        saved[i] = c->stream;
        c->stream = b->stream;
        if (c->opts.precision != HT_MIXED || c->opts.precond != HT_PREC_JACOBI) {
            for (int k = 0; k <= i; ++k) b->probs[k]->stream = saved[k];
            return bfail(b, HT_EINVAL, "batched problems need precision HT_MIXED with the Jacobi preconditioner");
        }
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, b->stream);
    int rc = HT_OK;
    std::vector<int> conv(np, 0), outer(np, 0), inner(np, 0);
    std::vector<double> res(np, 0.0);
    for (int i = 0; i < np && rc == HT_OK; ++i) rc = batch_head_begin(b->probs[i], dt);
    const double tol = b->probs[0]->opts.tol;
    const int max_outer = b->probs[0]->opts.max_outer > 0 ? b->probs[0]->opts.max_outer : 30;
    for (int k = 0; k <= max_outer && rc == HT_OK; ++k) {
        bool all = true;
        for (int i = 0; i < np && rc == HT_OK; ++i) {
            if (conv[i]) continue;
            rc = batch_outer_residual(b->probs[i], dt, tol, &conv[i], &res[i]);
            outer[i] = k;
            all = all && conv[i];
        }
        if (rc != HT_OK || all) break;
        if (k == max_outer) { rc = HT_ENOCONV; b->err = "batched head solve did not converge"; break; }
        for (int i = 0; i < np && rc == HT_OK; ++i) {
            ht_ctx* c = b->probs[i];
            const double base = c->opts.inner_tol > 0 ? c->opts.inner_tol : 1e-4;
            // no inner reduction beyond what the outer tolerance needs
            const double need = res[i] > 0 ? 0.5 * tol / res[i] : 1.0;
            const double itol = std::max(base, std::min(need, 0.5));
            rc = batch_inner_init(c, dt, conv[i] ? 1.0 : itol, c->opts.max_iter);
        }
        if (rc == HT_OK) {
            const ht_ctx* c0 = b->probs[0];
            rc = batch_inner_cg(b, dt, c0->opts.inner_tol > 0 ? c0->opts.inner_tol : 1e-4, c0->opts.max_iter);
        }
        for (int i = 0; i < np && rc == HT_OK; ++i) {
            if (conv[i]) continue;
            inner[i] += b->probs[i]->scal_host[1].iters;
            rc = batch_outer_update(b->probs[i]);
        }
    }
    cudaEventRecord(e1, b->stream);
    for (int i = 0; i < np; ++i) {
        ht_step_stats st{};
        int r2 = HT_OK;
        if (rc == HT_OK) r2 = batch_head_end_and_heat(b->probs[i], dt, &st);
        st.iters_head = inner[i];
        st.outer_head = outer[i];
        st.res_head = res[i];
        if (rc == HT_OK && r2 != HT_OK) {
            rc = r2;
            b->err = b->probs[i]->err;
        }
        if (stats) stats[i] = st;
    }
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (stats)
        for (int i = 0; i < np; ++i) stats[i].ms_head = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (int i = 0; i < np; ++i) b->probs[i]->stream = saved[i];
    return rc;
}

}  // extern "C"
