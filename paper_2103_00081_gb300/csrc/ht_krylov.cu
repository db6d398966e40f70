// Krylov solvers of the per-step linear systems: Jacobi- or Chebyshev-Jacobi-
// preconditioned CG for the symmetric head system (Eq. 3) and Jacobi-
// preconditioned BiCGStab for the nonsymmetric heat system (Eq. 4); plain
// FP64, or FP32 inner iterations inside an FP64 defect-correction loop.
//
// All scalars live on the device (struct Scal).  Vector kernels write one
// partial sum per CTA; a single-CTA scalar kernel reduces them in a fixed
// order and updates alpha / beta / omega, so every result is bitwise
// reproducible.  Kernels return at once when the solve is marked done, which
// lets the host enqueue several iterations between convergence checks.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>

#include <algorithm>

#include "ht_internal.cuh"

namespace ht {

int vec_grid(const ht_ctx* c) {
    const long long need = (c->grid.nn + kVecThreads - 1) / kVecThreads;
    long long g = (long long)(c->num_sms > 0 ? c->num_sms : 148) * kVecBlocksPerSM;
    if (need < g) g = need;
    return (int)(g < 1 ? 1 : g);
}

namespace {

__device__ __forceinline__ double bsum(double v) {
    __shared__ double ws[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) ws[wid] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? ws[lane] : 0.0;
    if (wid == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

// ---- scalar kernel ----------------------------------------------------------
enum {
    SC_CG_INIT, SC_CG_ALPHA, SC_CG_BETA, SC_FCG_BETA,
    SC_BI_INIT, SC_BI_ALPHA, SC_BI_OMEGA, SC_BI_BETA,
    SC_NORMS
};

__device__ double reduce_part(const double* part, int np) {
    double s = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) s += part[i];
    return bsum(s);
}

// part: [8][stride]; slot usage documented per opcode
__global__ void scalar_kernel(int op, const double* __restrict__ part, int stride, int np,
                              Scal* __restrict__ s, double tol2, int max_iter) {
    if (s->done && op != SC_NORMS) return;
    const double a0 = reduce_part(part + 0 * (size_t)stride, np);
    const double a1 = reduce_part(part + 1 * (size_t)stride, np);
    const double a2 = reduce_part(part + 2 * (size_t)stride, np);
    if (threadIdx.x != 0) return;
    switch (op) {
        case SC_CG_INIT:  // a0 = r.z, a1 = r.r, a2 = b.b
            s->tol2 = tol2; s->max_iter = max_iter;
            s->rz = a0; s->rr = a1; s->bb = a2; s->rr0 = a1;
            s->rz2[0] = a0;
            s->iters = 0; s->status = ST_OK;
            s->done = (a1 <= tol2 * a2 || a2 == 0.0) ? 1 : 0;
            if (!isfinite(a0) || !isfinite(a1)) { s->status = ST_NAN; s->done = 1; }
            break;
        case SC_CG_ALPHA:  // a0 = p.Ap
            s->pq = a0;
            if (!(a0 > 0.0) || !isfinite(a0)) { s->status = ST_BREAKDOWN; s->done = 1; break; }
            s->alpha = s->rz / a0;
            break;
        case SC_CG_BETA:  // a1 = r.z (new), a2 = r.r
            s->rz_new = a1; s->rr = a2;
            s->beta = a1 / s->rz;
            s->rz = a1;
            s->iters += 1;
            if (!isfinite(a1) || !isfinite(a2)) { s->status = ST_NAN; s->done = 1; }
            else if (a2 <= tol2 * s->bb || s->iters >= max_iter) s->done = 1;
            break;
        case SC_FCG_BETA:  // a0 = z.q, a1 = r.z (new), a2 = r.r; Polak-Ribiere beta
            s->rz_new = a1; s->rr = a2;
            s->beta = -s->alpha * a0 / s->rz;
            s->rz = a1;
            s->iters += 1;
            if (!isfinite(a1) || !isfinite(a2)) { s->status = ST_NAN; s->done = 1; }
            else if (a2 <= tol2 * s->bb || s->iters >= max_iter) s->done = 1;
            break;
        case SC_BI_INIT:  // a0 = rh.r, a1 = r.r, a2 = b.b
            s->tol2 = tol2; s->max_iter = max_iter;
            s->rho = a0; s->rr = a1; s->bb = a2; s->rr0 = a1;
            s->alpha = 1.0; s->omega = 1.0; s->beta = 0.0;
            s->iters = 0; s->status = ST_OK;
            s->done = (a1 <= tol2 * a2 || a2 == 0.0) ? 1 : 0;
            if (!isfinite(a0) || !isfinite(a1)) { s->status = ST_NAN; s->done = 1; }
            break;
        case SC_BI_ALPHA:  // a0 = rh.v
            s->rv = a0;
            if (a0 == 0.0 || !isfinite(a0)) { s->status = ST_BREAKDOWN; s->done = 1; break; }
            s->alpha = s->rho / a0;
            break;
        case SC_BI_OMEGA:  // a0 = t.s, a1 = t.t, a2 = s.s
            s->ts = a0; s->tt = a1;
            if (a1 == 0.0) {  // s = 0 exactly: x += alpha ph is the solution
                s->omega = 0.0;
            } else {
                s->omega = a0 / a1;
            }
            break;
        case SC_BI_BETA: {  // a0 = rh.r (new), a1 = r.r
            s->rr = a1;
            s->iters += 1;
            if (!isfinite(a0) || !isfinite(a1)) { s->status = ST_NAN; s->done = 1; break; }
            if (a1 <= tol2 * s->bb || s->iters >= max_iter) { s->done = 1; break; }
            if (a0 == 0.0 || s->omega == 0.0) { s->status = ST_BREAKDOWN; s->done = 1; break; }
            s->beta = (a0 / s->rho) * (s->alpha / s->omega);
            s->rho = a0;
            break;
        }
        case SC_NORMS:  // a0 = r.r, a1 = b.b
            s->rr = a0; s->bb = a1;
            break;
    }
}

// ---- vector kernels -----------------------------------------------------------
#define GRID_LOOP(i, n) \
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

template <typename T>
__device__ __forceinline__ void write3(double* part, int stride, T v0, T v1, T v2) {
    const double s0 = bsum((double)v0);
    const double s1 = bsum((double)v1);
    const double s2 = bsum((double)v2);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = s0;
        part[stride + blockIdx.x] = s1;
        part[2 * stride + blockIdx.x] = s2;
    }
}

// r = b - q; z = Dinv r; p = z.  part: r.z, r.r, b.b
template <typename T>
__global__ void cg_init_kernel(long long n, const T* __restrict__ b, const T* __restrict__ q,
                               const T* __restrict__ Dinv, T* __restrict__ r, T* __restrict__ p,
                               double* __restrict__ part, int stride) {
    T rz = 0, rr = 0, bb = 0;
    GRID_LOOP(i, n) {
        const T bi = b[i];
        const T ri = bi - q[i];
        const T zi = Dinv[i] * ri;
        r[i] = ri;
        p[i] = zi;
        rz = fma(ri, zi, rz);
        rr = fma(ri, ri, rr);
        bb = fma(bi, bi, bb);
    }
    write3<T>(part, stride, rz, rr, bb);
}

// x += alpha p; r -= alpha q; z = Dinv r.  part[1] = r.z, part[2] = r.r
template <typename T>
__global__ void cg_update_kernel(long long n, T* __restrict__ x, T* __restrict__ r,
                                 const T* __restrict__ p, const T* __restrict__ q,
                                 const T* __restrict__ Dinv, const Scal* __restrict__ s,
                                 double* __restrict__ part, int stride) {
    if (s->done) return;
    const T alpha = (T)s->alpha;
    T rz = 0, rr = 0;
    GRID_LOOP(i, n) {
        x[i] = fma(alpha, p[i], x[i]);
        const T ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        rz = fma(ri, Dinv[i] * ri, rz);
        rr = fma(ri, ri, rr);
    }
    write3<T>(part, stride, T(0), rz, rr);
}

// p = Dinv r + beta p
template <typename T>
__global__ void cg_pupdate_kernel(long long n, const T* __restrict__ r, const T* __restrict__ Dinv,
                                  T* __restrict__ p, const Scal* __restrict__ s) {
    if (s->done) return;
    const T beta = (T)s->beta;
    GRID_LOOP(i, n) p[i] = fma(beta, p[i], Dinv[i] * r[i]);
}


// ---- fused CG iteration (Jacobi) ------------------------------------------------
// alpha and beta are reduced redundantly, in a fixed order, by every CTA of the
// kernel that needs them, so a CG iteration is three launches: apply (with
// the p.Ap partials), x/r update, p update.  r.z is double-buffered by the
// iteration parity so that the CTA that stores the new value never races the
// CTAs that still read the old one.
template <typename T>
__global__ void cgf_update_kernel(long long n, T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p,
                                  const T* __restrict__ q, const T* __restrict__ Dinv, Scal* __restrict__ s,
                                  double* __restrict__ part, int stride, int np, int par) {
    if (s->done) return;
    __shared__ double sh_alpha;
    const double pq = reduce_part(part, np);
    if (threadIdx.x == 0) sh_alpha = pq;
    __syncthreads();
    const double pqv = sh_alpha;
    if (!(pqv > 0.0) || !isfinite(pqv)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) { s->status = ST_BREAKDOWN; s->done = 1; }
        return;
    }
    const T alpha = (T)(s->rz2[par] / pqv);
    T rz = 0, rr = 0;
    GRID_LOOP(i, n) {
        x[i] = fma(alpha, p[i], x[i]);
        const T ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        rz = fma(ri, Dinv[i] * ri, rz);
        rr = fma(ri, ri, rr);
    }
    const double a = bsum((double)rz);
    const double b = bsum((double)rr);
    if (threadIdx.x == 0) {
        part[(size_t)stride + blockIdx.x] = a;
        part[(size_t)2 * stride + blockIdx.x] = b;
    }
}

template <typename T>
__global__ void cgf_pupdate_kernel(long long n, const T* __restrict__ r, const T* __restrict__ Dinv,
                                   T* __restrict__ p, Scal* __restrict__ s, const double* __restrict__ part,
                                   int stride, int np, int par, double tol2, int max_iter) {
    if (s->done) return;
    __shared__ double sh[2];
    const double rz = reduce_part(part + (size_t)stride, np);
    if (threadIdx.x == 0) sh[0] = rz;
    const double rr = reduce_part(part + (size_t)2 * stride, np);
    if (threadIdx.x == 0) sh[1] = rr;
    __syncthreads();
    const double rzn = sh[0], rrn = sh[1];
    const T beta = (T)(rzn / s->rz2[par]);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        s->rz2[par ^ 1] = rzn;
        s->rr = rrn;
        s->iters += 1;
        if (!isfinite(rzn) || !isfinite(rrn)) { s->status = ST_NAN; s->done = 1; }
        else if (rrn <= tol2 * s->bb || s->iters >= max_iter) s->done = 1;
    }
    GRID_LOOP(i, n) p[i] = fma(beta, p[i], Dinv[i] * r[i]);
}

// BiCGStab
// r = b - q; rh = r; p = v = 0.  part: rh.r, r.r, b.b
template <typename T>
__global__ void bi_init_kernel(long long n, const T* __restrict__ b, const T* __restrict__ q,
                               T* __restrict__ r, T* __restrict__ rh, T* __restrict__ p,
                               T* __restrict__ v, double* __restrict__ part, int stride) {
    T rr = 0, bb = 0;
    GRID_LOOP(i, n) {
        const T bi = b[i];
        const T ri = bi - q[i];
        r[i] = ri;
        rh[i] = ri;
        p[i] = T(0);
        v[i] = T(0);
        rr = fma(ri, ri, rr);
        bb = fma(bi, bi, bb);
    }
    write3<T>(part, stride, rr, rr, bb);
}

// p = r + beta (p - omega v); ph = Dinv p
template <typename T>
__global__ void bi_p_kernel(long long n, const T* __restrict__ r, T* __restrict__ p,
                            const T* __restrict__ v, const T* __restrict__ Dinv, T* __restrict__ ph,
                            const Scal* __restrict__ s) {
    if (s->done) return;
    const T beta = (T)s->beta, omega = (T)s->omega;
    GRID_LOOP(i, n) {
        const T pi = fma(beta, fma(-omega, v[i], p[i]), r[i]);
        p[i] = pi;
        ph[i] = Dinv[i] * pi;
    }
}

// part[0] = a.b
template <typename T>
__global__ void dot_kernel(long long n, const T* __restrict__ a, const T* __restrict__ b,
                           double* __restrict__ part, int stride, const Scal* __restrict__ s) {
    if (s && s->done) return;
    T d = 0;
    GRID_LOOP(i, n) d = fma(a[i], b[i], d);
    write3<T>(part, stride, d, T(0), T(0));
}

// s = r - alpha v; sh = Dinv s
template <typename T>
__global__ void bi_s_kernel(long long n, const T* __restrict__ r, const T* __restrict__ v,
                            const T* __restrict__ Dinv, T* __restrict__ sv, T* __restrict__ sh,
                            const Scal* __restrict__ s) {
    if (s->done) return;
    const T alpha = (T)s->alpha;
    GRID_LOOP(i, n) {
        const T si = fma(-alpha, v[i], r[i]);
        sv[i] = si;
        sh[i] = Dinv[i] * si;
    }
}

// part: t.s, t.t, s.s
template <typename T>
__global__ void bi_ts_kernel(long long n, const T* __restrict__ t, const T* __restrict__ sv,
                             double* __restrict__ part, int stride, const Scal* __restrict__ s) {
    if (s->done) return;
    T ts = 0, tt = 0, ss = 0;
    GRID_LOOP(i, n) {
        const T ti = t[i], si = sv[i];
        ts = fma(ti, si, ts);
        tt = fma(ti, ti, tt);
        ss = fma(si, si, ss);
    }
    write3<T>(part, stride, ts, tt, ss);
}

// x += alpha ph + omega sh; r = s - omega t.  part: rh.r, r.r
template <typename T>
__global__ void bi_xr_kernel(long long n, T* __restrict__ x, T* __restrict__ r,
                             const T* __restrict__ ph, const T* __restrict__ sh,
                             const T* __restrict__ sv, const T* __restrict__ t,
                             const T* __restrict__ rh, double* __restrict__ part, int stride,
                             const Scal* __restrict__ s) {
    if (s->done) return;
    const T alpha = (T)s->alpha, omega = (T)s->omega;
    T rhr = 0, rr = 0;
    GRID_LOOP(i, n) {
        x[i] = fma(alpha, ph[i], fma(omega, sh[i], x[i]));
        const T ri = fma(-omega, t[i], sv[i]);
        r[i] = ri;
        rhr = fma(rh[i], ri, rhr);
        rr = fma(ri, ri, rr);
    }
    write3<T>(part, stride, rhr, rr, T(0));
}


// ---- GMRES(m) ----------------------------------------------------------------
// Right-preconditioned restarted GMRES with Jacobi M = D: A D^-1 u = b,
// x = x0 + D^-1 V y.  Arnoldi by classical Gram-Schmidt applied twice (CGS2).
// The multi-dot runs on a 2D grid (node slices x chunks of kDotChunk basis
// vectors), the Hessenberg entries are reduced by one CTA each, Givens
// rotations and the triangular solve run in a single-CTA kernel.
enum { GM_INIT, GM_NORM, GM_SOLVE };
#define HIDX(j, k) ((j) + (kMaxRestart + 1) * (k))

// r = b - q into V_0; part: r.r, b.b
template <typename T>
__global__ void gm_init_kernel(long long n, const T* __restrict__ b, const T* __restrict__ q,
                               T* __restrict__ v0, double* __restrict__ part, int stride) {
    T rr = 0, bb = 0;
    GRID_LOOP(i, n) {
        const T bi = b[i];
        const T ri = bi - q[i];
        v0[i] = ri;
        rr = fma(ri, ri, rr);
        bb = fma(bi, bi, bb);
    }
    write3<T>(part, stride, rr, bb, T(0));
}

// V_k *= inv; z = Dinv V_k
template <typename T>
__global__ void gm_prep_kernel(long long n, T* __restrict__ vk, const T* __restrict__ Dinv,
                               T* __restrict__ z, const Gmres* __restrict__ gm, const Scal* __restrict__ s) {
    if (s->done) return;
    const T inv = (T)gm->inv;
    GRID_LOOP(i, n) {
        const T v = vk[i] * inv;
        vk[i] = v;
        z[i] = Dinv[i] * v;
    }
}

// part[j*stride + bx] = partial of V_j . w for j in chunk blockIdx.y (j <= k)
template <typename T>
__global__ void gm_dots_kernel(long long n, const T* __restrict__ V, long long ldv, int k,
                               const T* __restrict__ w, double* __restrict__ part, int stride,
                               const Scal* __restrict__ s) {
    if (s->done) return;
    const int j0 = blockIdx.y * kDotChunk;
    const int cnt = min(kDotChunk, k + 1 - j0);
    T acc[kDotChunk];
#pragma unroll
    for (int j = 0; j < kDotChunk; ++j) acc[j] = T(0);
    const T* Vc = V + (size_t)j0 * ldv;
    GRID_LOOP(i, n) {
        const T wi = w[i];
#pragma unroll
        for (int j = 0; j < kDotChunk; ++j)
            if (j < cnt) acc[j] = fma(Vc[j * ldv + i], wi, acc[j]);
    }
    __shared__ double ws[32][kDotChunk + 1];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int j = 0; j < kDotChunk; ++j) {
        if (j < cnt) {
            double v = (double)acc[j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) ws[wid][j] = v;
        }
    }
    __syncthreads();
    if ((int)threadIdx.x < cnt) {
        double sum = 0.0;
        for (int w2 = 0; w2 < nw; ++w2) sum += ws[w2][threadIdx.x];
        part[(size_t)(j0 + threadIdx.x) * stride + blockIdx.x] = sum;
    }
}

// one CTA per Hessenberg entry j: pass 1 sets H[j][k], pass 2 adds the
// reorthogonalisation correction hc[j]
__global__ void gm_hreduce_kernel(const double* __restrict__ part, int stride, int np, Gmres* __restrict__ gm,
                                  int k, int pass, const Scal* __restrict__ s) {
    if (s->done) return;
    const int j = blockIdx.x;
    const double v = reduce_part(part + (size_t)j * stride, np);
    if (threadIdx.x == 0) {
        if (pass == 1) {
            gm->H[HIDX(j, k)] = v;
        } else {
            gm->hc[j] = v;
            gm->H[HIDX(j, k)] += v;
        }
    }
}

// w -= sum_{j<=k} c_j V_j with c = H[:,k] (pass 1) or hc (pass 2); pass 2 also
// writes the partial of |w|^2 into slot 0.
template <typename T>
__global__ void gm_orth_kernel(long long n, const T* __restrict__ V, long long ldv, int k, T* __restrict__ w,
                               const Gmres* __restrict__ gm, int pass, double* __restrict__ part, int stride,
                               const Scal* __restrict__ s) {
    if (s->done) return;
    __shared__ T cf[kMaxRestart + 1];
    for (int j = threadIdx.x; j <= k; j += blockDim.x) cf[j] = (T)(pass == 1 ? gm->H[HIDX(j, k)] : gm->hc[j]);
    __syncthreads();
    T ww = 0;
    GRID_LOOP(i, n) {
        T v = w[i];
        int j = 0;
        for (; j + 3 <= k; j += 4) {
            v = fma(-cf[j], V[(size_t)j * ldv + i], v);
            v = fma(-cf[j + 1], V[(size_t)(j + 1) * ldv + i], v);
            v = fma(-cf[j + 2], V[(size_t)(j + 2) * ldv + i], v);
            v = fma(-cf[j + 3], V[(size_t)(j + 3) * ldv + i], v);
        }
        for (; j <= k; ++j) v = fma(-cf[j], V[(size_t)j * ldv + i], v);
        w[i] = v;
        ww = fma(v, v, ww);
    }
    if (pass == 2) write3<T>(part, stride, ww, T(0), T(0));
}

// x += Dinv (V y)
template <typename T>
__global__ void gm_update_kernel(long long n, const T* __restrict__ V, long long ldv, const Gmres* __restrict__ gm,
                                 const Scal* __restrict__ s, const T* __restrict__ Dinv, T* __restrict__ x) {
    const int kd = s->kdone;
    __shared__ T y[kMaxRestart];
    for (int j = threadIdx.x; j < kd; j += blockDim.x) y[j] = (T)gm->y[j];
    __syncthreads();
    GRID_LOOP(i, n) {
        T u = 0;
        for (int j = 0; j < kd; ++j) u = fma(y[j], V[(size_t)j * ldv + i], u);
        x[i] = fma(Dinv[i], u, x[i]);
    }
}

__global__ void gm_scalar_kernel(int op, int k, const double* __restrict__ part, int stride, int np,
                                 Scal* __restrict__ s, Gmres* __restrict__ gm, double tol2, int max_iter, int m) {
    if (op == GM_NORM && s->done) return;
    __shared__ double red[2];
    const int cnt = op == GM_INIT ? 2 : (op == GM_NORM ? 1 : 0);
    for (int j = 0; j < cnt; ++j) {
        const double v = reduce_part(part + (size_t)j * stride, np);
        if (threadIdx.x == 0) red[j] = v;
    }
    if (op == GM_SOLVE) {
        // back substitution, one row at a time; the row update is shared by the CTA
        const int kd = s->kdone;
        __shared__ double yi;
        for (int i = kd - 1; i >= 0; --i) {
            double t = 0.0;
            for (int j = i + 1 + threadIdx.x; j < kd; j += blockDim.x) t += gm->H[HIDX(i, j)] * gm->y[j];
            t = bsum(t);
            if (threadIdx.x == 0) {
                yi = (gm->g[i] - t) / gm->H[HIDX(i, i)];
                gm->y[i] = yi;
            }
            __syncthreads();
        }
        return;
    }
    if (threadIdx.x != 0) return;
    switch (op) {
        case GM_INIT: {
            const double rr = red[0], bb = red[1];
            s->rr = rr; s->bb = bb; s->rr0 = rr;
            s->kdone = 0; s->status = ST_OK;
            const double beta = sqrt(rr);
            gm->g[0] = beta;
            gm->inv = beta > 0 ? 1.0 / beta : 0.0;
            s->conv = (rr <= tol2 * bb || bb == 0.0) ? 1 : 0;
            s->done = s->conv;
            if (!isfinite(rr)) { s->status = ST_NAN; s->done = 1; }
            break;
        }
        case GM_NORM: {
            const double hk1 = sqrt(red[0]);
            for (int i = 0; i < k; ++i) {
                const double a = gm->H[HIDX(i, k)], b = gm->H[HIDX(i + 1, k)];
                gm->H[HIDX(i, k)] = gm->cs[i] * a + gm->sn[i] * b;
                gm->H[HIDX(i + 1, k)] = -gm->sn[i] * a + gm->cs[i] * b;
            }
            const double a = gm->H[HIDX(k, k)], b = hk1;
            const double r = hypot(a, b);
            const double cs = r > 0 ? a / r : 1.0, sn = r > 0 ? b / r : 0.0;
            gm->cs[k] = cs; gm->sn[k] = sn;
            gm->H[HIDX(k, k)] = r;
            gm->H[HIDX(k + 1, k)] = 0.0;
            gm->g[k + 1] = -sn * gm->g[k];
            gm->g[k] = cs * gm->g[k];
            gm->inv = hk1 > 0 ? 1.0 / hk1 : 0.0;
            s->rr = gm->g[k + 1] * gm->g[k + 1];
            s->kdone = k + 1;
            s->iters += 1;
            if (!isfinite(s->rr) || !isfinite(r)) { s->status = ST_NAN; s->done = 1; break; }
            if (r == 0.0) { s->status = ST_BREAKDOWN; s->done = 1; s->kdone = k; break; }
            if (s->rr <= tol2 * s->bb || hk1 == 0.0) { s->conv = 1; s->done = 1; }
            else if (k + 1 >= m || s->iters >= max_iter) s->done = 1;
            break;
        }
    }
}


// ---- Chebyshev-Jacobi polynomial preconditioner ----------------------------------
// z = p_k(D^-1 A) D^-1 r: k steps of the Chebyshev iteration for A z = r from
// z = 0 on the interval [a, b] = [b / ratio, 1.2 lambda_max] of D^-1 A.  The
// residual polynomial R = T_k((theta - lambda) / delta) / T_k(theta / delta)
// lies in (-1, 1) for every lambda in (0, b] (below a the argument stays in
// (1, theta / delta)), so lambda p_k(lambda) = 1 - R > 0: the preconditioner
// is symmetric positive definite, as CG requires, and on [a, b] the
// preconditioned spectrum is within 1 -+ 1 / T_k(theta / delta).
template <typename T>
__global__ void cheb_init_kernel(long long n, const T* __restrict__ r, const T* __restrict__ Dinv,
                                 T* __restrict__ d, T* __restrict__ z, T inv_theta, const Scal* __restrict__ s) {
    if (s && s->done) return;
    GRID_LOOP(i, n) {
        const T v = Dinv[i] * r[i] * inv_theta;
        d[i] = v;
        z[i] = v;
    }
}

// d = c1 d + c2 Dinv (r - w); z += d
template <typename T>
__global__ void cheb_step_kernel(long long n, const T* __restrict__ r, const T* __restrict__ w,
                                 const T* __restrict__ Dinv, T* __restrict__ d, T* __restrict__ z, T c1, T c2,
                                 const Scal* __restrict__ s) {
    if (s && s->done) return;
    GRID_LOOP(i, n) {
        const T di = fma(c1, d[i], c2 * Dinv[i] * (r[i] - w[i]));
        d[i] = di;
        z[i] += di;
    }
}

// CG with an explicit preconditioned vector z:
// x += alpha p; r -= alpha q.  part[2] = r.r
template <typename T>
__global__ void cgz_update_kernel(long long n, T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p,
                                  const T* __restrict__ q, const Scal* __restrict__ s, double* __restrict__ part,
                                  int stride) {
    if (s->done) return;
    const T alpha = (T)s->alpha;
    T rr = 0;
    GRID_LOOP(i, n) {
        x[i] = fma(alpha, p[i], x[i]);
        const T ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        rr = fma(ri, ri, rr);
    }
    write3<T>(part, stride, T(0), T(0), rr);
}

// part[slot] = r.z (the other slots keep what the update / init wrote); with
// q != nullptr also part[0] = z.q for the flexible (Polak-Ribiere) beta
template <typename T>
__global__ void cgz_dot_kernel(long long n, const T* __restrict__ r, const T* __restrict__ z,
                               const T* __restrict__ q, double* __restrict__ part, int stride, int slot,
                               const Scal* __restrict__ s) {
    if (s->done) return;
    T rz = 0, zq = 0;
    GRID_LOOP(i, n) {
        const T zi = z[i];
        rz = fma(r[i], zi, rz);
        if (q) zq = fma(zi, q[i], zq);
    }
    const double v = bsum((double)rz);
    const double u = bsum((double)zq);
    if (threadIdx.x == 0) {
        part[(size_t)slot * stride + blockIdx.x] = v;
        if (q) part[blockIdx.x] = u;
    }
}

// p = z + beta p
template <typename T>
__global__ void cgz_pupdate_kernel(long long n, const T* __restrict__ z, T* __restrict__ p,
                                   const Scal* __restrict__ s) {
    if (s->done) return;
    const T beta = (T)s->beta;
    GRID_LOOP(i, n) p[i] = fma(beta, p[i], z[i]);
}

// r = b - q, z-independent init: part: 0, r.r, b.b  (r.z comes from cgz_dot)
template <typename T>
__global__ void cgz_init_kernel(long long n, const T* __restrict__ b, const T* __restrict__ q,
                                T* __restrict__ r, double* __restrict__ part, int stride) {
    T rr = 0, bb = 0;
    GRID_LOOP(i, n) {
        const T bi = b[i];
        const T ri = bi - q[i];
        r[i] = ri;
        rr = fma(ri, ri, rr);
        bb = fma(bi, bi, bb);
    }
    write3<T>(part, stride, T(0), rr, bb);
}

template <typename T>
__global__ void copy_kernel(long long n, const T* __restrict__ a, T* __restrict__ b) {
    GRID_LOOP(i, n) b[i] = a[i];
}

// power iteration on D^-1 A: v = D^-1 w / |.|, part[0] = |D^-1 w|^2, part[1] = v.v
__global__ void power_kernel(long long n, const double* __restrict__ w, const double* __restrict__ Dinv,
                             double* __restrict__ v, double inv_norm, double* __restrict__ part, int stride) {
    double a = 0, b = 0;
    GRID_LOOP(i, n) {
        const double vi = Dinv[i] * w[i] * inv_norm;
        v[i] = vi;
        a = fma(vi, vi, a);
    }
    write3<double>(part, stride, a, b, 0.0);
}

__global__ void seed_kernel(long long n, double* __restrict__ v) {
    GRID_LOOP(i, n) {
        unsigned long long z = (unsigned long long)i * 0x9E3779B97F4A7C15ULL + 0x632BE59BD9B4E019ULL;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        z ^= z >> 31;
        v[i] = 2.0 * (double)(z >> 11) * (1.0 / 9007199254740992.0) - 1.0;   // zero-mean, all frequencies
    }
}

// ---- mixed precision helpers ---------------------------------------------------
// r = b - q (FP64); r32 = (float) r.  part: r.r, b.b
__global__ void resid_kernel(long long n, const double* __restrict__ b, const double* __restrict__ q,
                             double* __restrict__ r, float* __restrict__ r32,
                             double* __restrict__ part, int stride) {
    double rr = 0, bb = 0;
    GRID_LOOP(i, n) {
        const double bi = b[i];
        const double ri = bi - q[i];
        if (r) r[i] = ri;
        if (r32) r32[i] = (float)ri;
        rr = fma(ri, ri, rr);
        bb = fma(bi, bi, bb);
    }
    write3<double>(part, stride, rr, bb, 0.0);
}

// r = b - q with q from the FP32 operator: r32 = (float) r, partials r.r, b.b
// r32 = b - q with q = A x from the FP32 operator.  On Dirichlet rows the
// constrained operator is the identity, so the residual there is taken as
// b - x in FP64 (zero once x carries the Dirichlet values): the FP32 copy of
// x_D would leave a rounding residual on rows that the fused Krylov
// iterations keep at zero and could never reduce.
__global__ void resid32_kernel(const Grid g, long long n, const double* __restrict__ b, const float* __restrict__ q,
                               const double* __restrict__ x, float* __restrict__ r32, double* __restrict__ part,
                               int stride) {
    double rr = 0, bb = 0;
    const long long nxy = (long long)g.Nx * g.Ny;
    GRID_LOOP(i, n) {
        const double bi = b[i];
        bool d = false;
        if (g.dmask) {
            const int k = (int)(i / nxy);
            const int m = (int)(i - (long long)k * nxy);
            const int jj = m / g.Nx, ii = m - jj * g.Nx;
            const int dm = g.dmask;
            d = ((dm & 1) && ii == 0) || ((dm & 2) && ii == g.Nx - 1) || ((dm & 4) && jj == 0) ||
                ((dm & 8) && jj == g.Ny - 1) || ((dm & 16) && k == 0) || ((dm & 32) && k == g.Nz - 1);
        }
        const double ri = d ? bi - x[i] : bi - (double)q[i];
        r32[i] = (float)ri;
        rr = fma(ri, ri, rr);
        bb = fma(bi, bi, bb);
    }
    write3<double>(part, stride, rr, bb, 0.0);
}

__global__ void to_f32_kernel(long long n, const double* __restrict__ a, float* __restrict__ b) {
    GRID_LOOP(i, n) b[i] = (float)a[i];
}

__global__ void add_f32_kernel(long long n, double* __restrict__ x, const float* __restrict__ d) {
    GRID_LOOP(i, n) x[i] += (double)d[i];
}

template <typename T>
__global__ void fill_kernel(long long n, T* __restrict__ x, T v) {
    GRID_LOOP(i, n) x[i] = v;
}

// Dinv = 1 / D in both precisions
__global__ void inv_kernel(long long n, const double* __restrict__ D, double* __restrict__ Dinv,
                           float* __restrict__ Dinv32) {
    GRID_LOOP(i, n) {
        const double v = 1.0 / D[i];
        Dinv[i] = v;
        Dinv32[i] = (float)v;
    }
}

__global__ void dirichlet_kernel(const Grid g, const double* __restrict__ gv, double* __restrict__ x) {
    GRID_LOOP(id, g.nn) {
        const int i = (int)(id % g.Nx);
        const int j = (int)((id / g.Nx) % g.Ny);
        const int k = (int)(id / ((long long)g.Nx * g.Ny));
        const int m = g.dmask;
        const bool d = ((m & 1) && i == 0) || ((m & 2) && i == g.Nx - 1) || ((m & 4) && j == 0) ||
                       ((m & 8) && j == g.Ny - 1) || ((m & 16) && k == 0) || ((m & 32) && k == g.Nz - 1);
        if (d) x[id] = gv[id];
    }
}

// ---- host drivers -------------------------------------------------------------
int sync_scal(ht_ctx* c, int slot) {
    HT_CUDA(c, cudaMemcpyAsync(c->scal_host + slot, c->scal + slot, sizeof(Scal), cudaMemcpyDeviceToHost,
                               c->stream));
    HT_CUDA(c, cudaStreamSynchronize(c->stream));
    return HT_OK;
}

int scalar(ht_ctx* c, int op, int np, int slot, double tol, int max_iter) {
    scalar_kernel<<<1, 256, 0, c->stream>>>(op, c->part, c->part_stride, np, c->scal + slot, tol * tol,
                                            max_iter); ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    return HT_OK;
}

struct Vecs64 {
    double *x, *r, *p, *q, *Dinv, *rh, *v, *s, *t, *ph, *sh;
};
struct Vecs32 {
    float *x, *r, *p, *q, *Dinv, *rh, *v, *s, *t, *ph, *sh;
};

template <typename T>
int apply_T(ht_ctx* c, int field, double dt, const T* x, T* y, double* part, int* np, const Scal* sc);
template <>
int apply_T<double>(ht_ctx* c, int field, double dt, const double* x, double* y, double* part, int* np,
                    const Scal* sc) {
    return launch_apply64(c, field, dt, x, y, part, np, sc);
}
template <>
int apply_T<float>(ht_ctx* c, int field, double dt, const float* x, float* y, double* part, int* np,
                   const Scal* sc) {
    return launch_apply32(c, field, (float)dt, x, y, part, np, sc);
}

inline int fused_cg_iteration(ht_ctx* c, double dt, const Vecs64& w, Scal* sc, int first) {
    return fused_cg_iteration64(c, dt, w.x, w.r, w.Dinv, w.p, sc, first);
}
inline int fused_cg_iteration(ht_ctx* c, double dt, const Vecs32& w, Scal* sc, int first) {
    return fused_cg_iteration32(c, (float)dt, w.x, w.r, w.Dinv, w.p, sc, first);
}
inline int fused_bicgstab_iteration(ht_ctx* c, double dt, const Vecs64& w, Scal* sc) {
    return fused_bicgstab_iteration64(c, dt, w.x, w.r, w.rh, w.p, w.v, w.t, w.Dinv, sc);
}
inline int fused_bicgstab_iteration(ht_ctx* c, double dt, const Vecs32& w, Scal* sc) {
    return fused_bicgstab_iteration32(c, (float)dt, w.x, w.r, w.rh, w.p, w.v, w.t, w.Dinv, sc);
}

// Fused iterations per CUDA graph replay.
constexpr int kGraphIters = 8;

// Capture kGraphIters calls of iter() into gr (kernel launches only; the
// context's launch counter is restored, replays count their launches).
template <class Iter>
int capture_fused(ht_ctx* c, ht_ctx::FusedGraph& gr, Iter&& iter) {
    if (gr.exec) { cudaGraphExecDestroy(gr.exec); gr.exec = nullptr; }
    const long long nl = c->n_launch;
    HT_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    int rc = HT_OK;
    for (int k = 0; k < kGraphIters && rc == HT_OK; ++k) rc = iter();
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
    c->n_launch = nl;
    if (rc != HT_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        if (rc != HT_OK) return rc;
        HT_CUDA(c, e);
    }
    const cudaError_t ie = cudaGraphInstantiate(&gr.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) { gr.exec = nullptr; HT_CUDA(c, ie); }
    return HT_OK;
}

// Drive fused Krylov iterations until the device flags convergence.  iter(1)
// is the first iteration, iter(0) every later one.  With graphs on, later
// iterations are replays of a graph of kGraphIters iterations, captured once
// per key (the vectors, the step size and the operator scalars); iterations
// launched after convergence return at once.  The host checks convergence
// every 8..64 iterations.  When profiling, each check interval is timed with
// CUDA events and kept only if every iteration in it did work (counted per
// iteration in ht_profile_read).
template <class Iter>
int drive_fused(ht_ctx* c, int slot, ht_ctx::FusedGraph& gr, const void* const* key, int nkey, double dt,
                int kind, int launches_per_iter, Iter&& iter) {
    HT_TRY(iter(1));
    bool graphs = c->opts.use_graphs != 0;
    if (graphs) {
        bool same = gr.exec != nullptr && gr.dt == dt;
        for (int k = 0; k < nkey && same; ++k) same = gr.key[k] == key[k];
        if (!same) {
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(c->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
                cudaGetLastError();
                graphs = false;       // the caller is capturing this stream: launch directly
            } else {
                HT_TRY(capture_fused(c, gr, [&] { return iter(0); }));
                for (int k = 0; k < nkey; ++k) gr.key[k] = key[k];
                gr.dt = dt;
            }
        }
    }
    int chunk = c->opts.check_every > 0 ? c->opts.check_every : 8;
    if (graphs) chunk = (chunk + kGraphIters - 1) / kGraphIters * kGraphIters;
    const int base_chunk = chunk;
    // with a count from the previous step, the first check comes a few
    // iterations before it, then every base_chunk (doubling) iterations
    if (c->cur_hint > 0) {
        int h = c->cur_hint - 1 - 8;
        if (graphs) h = h / kGraphIters * kGraphIters;
        if (h > chunk) chunk = h;
    }
    HT_TRY(sync_scal(c, slot));
    bool first_chunk = true;
    while (!c->scal_host[slot].done) {
        const int before = c->scal_host[slot].iters;
        if (c->prof_on) HT_TRY(prof_begin(c, kind));
        if (graphs) {
            for (int k = 0; k < chunk; k += kGraphIters) {
                HT_CUDA(c, cudaGraphLaunch(gr.exec, c->stream));
                c->n_launch += (long long)kGraphIters * launches_per_iter;
            }
        } else {
            for (int k = 0; k < chunk; ++k) HT_TRY(iter(0));
        }
        if (c->prof_on) HT_TRY(prof_end_weighted(c, chunk));
        HT_TRY(sync_scal(c, slot));
        if (c->prof_on && c->scal_host[slot].iters - before != chunk) prof_drop_last(c);
        if (first_chunk && chunk > base_chunk) chunk = base_chunk;
        else if (chunk < 64) chunk *= 2;
        first_chunk = false;
    }
    return HT_OK;
}

// Preconditioned CG on A0 x = b (x holds the initial guess).  Returns
// iterations in *iters; status in c->scal[slot].
template <typename T, class V>
int run_cg(ht_ctx* c, double dt, const V& w, const T* b, int slot, double tol, int max_iter, int* iters) {
    const long long n = c->grid.nn;
    const int G = vec_grid(c);
    const int S = c->part_stride;
    Scal* sc = c->scal + slot;
    int np = 0;
    HT_TRY(apply_T<T>(c, HT_HEAD, dt, w.x, w.q, nullptr, nullptr, nullptr));
    cg_init_kernel<T><<<G, kVecThreads, 0, c->stream>>>(n, b, w.q, w.Dinv, w.r, w.p, c->part, S); ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    HT_CUDA(c, cudaMemsetAsync(sc, 0, sizeof(Scal), c->stream));
    HT_TRY(scalar(c, SC_CG_INIT, G, slot, tol, max_iter));
    int chunk = c->opts.check_every > 0 ? c->opts.check_every : 8;
    HT_TRY(sync_scal(c, slot));
    if (c->scal_host[slot].bb == 0.0) {  // b = 0: the solution is x = 0
        fill_kernel<T><<<G, kVecThreads, 0, c->stream>>>(n, w.x, T(0)); ++c->n_launch;
        HT_CUDA(c, cudaGetLastError());
        *iters = 0;
        return HT_OK;
    }
    int it_enq = 0;
    if (sizeof(T) == 4 && q1_cg_available(c, 1)) {
        // one launch per iteration (single-reduction CG on Q1 tiles); the
        // first launch only forms alpha_0 = r.z / z.Az.  Launch j reads r, p
        // from copy j % 2 and writes copy (j + 1) % 2 (copy 1 of r is s, of p
        // is q, both free in the head CG); graphs hold an even number of
        // launches, so every replay starts on the same copy
        const double ss = c->Ss;
        float* rr[2] = {(float*)w.r, (float*)w.s};
        float* pp[2] = {(float*)w.p, (float*)w.q};
        const void* key[6] = {w.x, w.r, w.p, w.s, w.q, sc};
        ht_ctx::FusedGraph& gr = c->g_cg1;
        if (gr.exec && gr.ss != ss) gr.dt = -1.0;
        long long j = 0;
        HT_TRY(drive_fused(c, slot, gr, key, 6, dt, HT_PROF_CG_ITER, 1, [&](int first) {
            const int a = (int)(j & 1);
            ++j;
            return q1_cg_iteration32(c, (float)dt, (float*)w.x, rr[a], pp[a], rr[a ^ 1], pp[a ^ 1], sc, first);
        }));
        gr.ss = ss;
        *iters = c->scal_host[slot].iters;
        return HT_OK;
    }
    if (fused_cg_available(c, sizeof(T) == 4)) {
        // two launches per iteration: the p update rides in the element pass,
        // the x / r update and the next dot products in the node gather
        const double ss = c->Ss;
        const void* key[5] = {w.x, w.r, w.Dinv, w.p, sc};
        ht_ctx::FusedGraph& gr = c->g_cg[sizeof(T) == 4];
        if (gr.exec && gr.ss != ss) gr.dt = -1.0;   // operator scalar changed: recapture
        HT_TRY(drive_fused(c, slot, gr, key, 5, dt, HT_PROF_CG_ITER, 2,
                           [&](int first) { return fused_cg_iteration(c, dt, w, sc, first); }));
        gr.ss = ss;
        *iters = c->scal_host[slot].iters;
        return HT_OK;
    }
    while (!c->scal_host[slot].done) {
        for (int k = 0; k < chunk; ++k, ++it_enq) {
            const int par = it_enq & 1;
            HT_TRY(apply_T<T>(c, HT_HEAD, dt, w.p, w.q, c->part, &np, sc));
            cgf_update_kernel<T><<<G, kVecThreads, 0, c->stream>>>(n, w.x, w.r, w.p, w.q, w.Dinv, sc, c->part, S, np,
                                                                   par); ++c->n_launch;
            cgf_pupdate_kernel<T><<<G, kVecThreads, 0, c->stream>>>(n, w.r, w.Dinv, w.p, sc, c->part, S, G, par,
                                                                    tol * tol, max_iter); ++c->n_launch;
        }
        HT_CUDA(c, cudaGetLastError());
        HT_TRY(sync_scal(c, slot));
        if (chunk < 64) chunk *= 2;
    }
    *iters = c->scal_host[slot].iters;
    return HT_OK;
}

template <typename T, class V>
int run_bicgstab(ht_ctx* c, double dt, const V& w, const T* b, int slot, double tol, int max_iter,
                 int* iters) {
    const long long n = c->grid.nn;
    const int G = vec_grid(c);
    const int S = c->part_stride;
    Scal* sc = c->scal + slot;
    int total = 0;
    for (int restart = 0; restart < 3; ++restart) {
        HT_TRY(apply_T<T>(c, HT_TEMP, dt, w.x, w.q, nullptr, nullptr, nullptr));
        bi_init_kernel<T><<<G, kVecThreads, 0, c->stream>>>(n, b, w.q, w.r, w.rh, w.p, w.v, c->part, S); ++c->n_launch;
        HT_CUDA(c, cudaGetLastError());
        HT_CUDA(c, cudaMemsetAsync(sc, 0, sizeof(Scal), c->stream));
        HT_TRY(scalar(c, SC_BI_INIT, G, slot, tol, max_iter - total));
        HT_TRY(sync_scal(c, slot));
        if (c->scal_host[slot].bb == 0.0) {
            fill_kernel<T><<<G, kVecThreads, 0, c->stream>>>(n, w.x, T(0)); ++c->n_launch;
            HT_CUDA(c, cudaGetLastError());
            break;
        }
        int chunk = c->opts.check_every > 0 ? c->opts.check_every : 8;
        // the fused heat kernels treat the face Dirichlet rows only
        const bool q1 = sizeof(T) == 4 && q1_bicgstab_available(c) && heat_fused_ok(c);
        const bool fused = q1 || (fused_cg_available(c, sizeof(T) == 4) && heat_fused_ok(c));
        if (q1) {
            // two tiled heat applies and the update per iteration; iteration j
            // reads p, v from copy j % 2 and writes copy (j + 1) % 2 (copy 1 is
            // ph, sh, free in the fused iteration); graphs hold an even number
            // of iterations, so every replay starts on the same copy
            const double ss = c->cT_u + 3.0 * c->lam_u + 7.0 * c->cw;
            float* pp[2] = {(float*)w.p, (float*)w.ph};
            float* vv[2] = {(float*)w.v, (float*)w.sh};
            const void* key[10] = {w.x, w.r, w.rh, w.p, w.v, w.ph, w.sh, w.t, w.Dinv, sc};
            ht_ctx::FusedGraph& gr = c->g_bi1;
            if (gr.exec && gr.ss != ss) gr.dt = -1.0;
            long long j = 0;
            HT_TRY(drive_fused(c, slot, gr, key, 10, dt, HT_PROF_BICGSTAB_ITER, 3, [&](int) {
                const int a = (int)(j & 1);
                ++j;
                return q1_bicgstab_iteration32(c, (float)dt, (float*)w.x, (float*)w.r, (const float*)w.rh, pp[a],
                                               vv[a], pp[a ^ 1], vv[a ^ 1], (float*)w.t, (const float*)w.Dinv, sc);
            }));
            gr.ss = ss;
        } else if (fused) {
            // five launches per iteration (two element / node pass pairs and
            // the update); the first iteration needs no special form
            const double ss = c->cT_u + 3.0 * c->lam_u + 7.0 * c->cw;
            const void* key[8] = {w.x, w.r, w.rh, w.p, w.v, w.t, w.Dinv, sc};
            ht_ctx::FusedGraph& gr = c->g_bi[sizeof(T) == 4];
            if (gr.exec && gr.ss != ss) gr.dt = -1.0;
            HT_TRY(drive_fused(c, slot, gr, key, 8, dt, HT_PROF_BICGSTAB_ITER, 5,
                               [&](int) { return fused_bicgstab_iteration(c, dt, w, sc); }));
            gr.ss = ss;
        }
        while (!c->scal_host[slot].done) {
            for (int k = 0; !fused && k < chunk; ++k) {
                bi_p_kernel<T><<<G, kVecThreads, 0, c->stream>>>(n, w.r, w.p, w.v, w.Dinv, w.ph, sc); ++c->n_launch;
                HT_TRY(apply_T<T>(c, HT_TEMP, dt, w.ph, w.v, nullptr, nullptr, sc));
                dot_kernel<T><<<G, kVecThreads, 0, c->stream>>>(n, w.rh, w.v, c->part, S, sc); ++c->n_launch;
                HT_TRY(scalar(c, SC_BI_ALPHA, G, slot, tol, max_iter - total));
                bi_s_kernel<T><<<G, kVecThreads, 0, c->stream>>>(n, w.r, w.v, w.Dinv, w.s, w.sh, sc); ++c->n_launch;
                HT_TRY(apply_T<T>(c, HT_TEMP, dt, w.sh, w.t, nullptr, nullptr, sc));
                bi_ts_kernel<T><<<G, kVecThreads, 0, c->stream>>>(n, w.t, w.s, c->part, S, sc); ++c->n_launch;
                HT_TRY(scalar(c, SC_BI_OMEGA, G, slot, tol, max_iter - total));
                bi_xr_kernel<T><<<G, kVecThreads, 0, c->stream>>>(n, w.x, w.r, w.ph, w.sh, w.s, w.t, w.rh,
                                                                  c->part, S, sc); ++c->n_launch;
                HT_TRY(scalar(c, SC_BI_BETA, G, slot, tol, max_iter - total));
            }
            HT_CUDA(c, cudaGetLastError());
            HT_TRY(sync_scal(c, slot));
            if (chunk < 32) chunk *= 2;
        }
        total += c->scal_host[slot].iters;
        if (c->scal_host[slot].status != ST_BREAKDOWN) break;
        // breakdown: restart from the current iterate with a fresh shadow residual
    }
    *iters = total;
    return HT_OK;
}


template <typename T>
T* gm_basis(ht_ctx* c);
template <>
double* gm_basis<double>(ht_ctx* c) { return c->V64; }
template <>
float* gm_basis<float>(ht_ctx* c) { return c->V32; }

int ensure_basis(ht_ctx* c, int m, bool fp32) {
    const size_t n = (size_t)c->grid.nn * (m + 1);
    if (c->V_m >= m + 1 && (fp32 ? c->V32 != nullptr : c->V64 != nullptr)) return HT_OK;
    if (c->V_m < m + 1) {
        if (c->V64) cudaFree(c->V64);
        if (c->V32) cudaFree(c->V32);
        c->V64 = nullptr;
        c->V32 = nullptr;
        c->V_m = m + 1;
    }
    cudaError_t e = fp32 ? cudaMalloc(&c->V32, n * sizeof(float)) : cudaMalloc(&c->V64, n * sizeof(double));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, HT_ENOMEM, "GMRES basis of %d vectors does not fit", m + 1);
    }
    return HT_OK;
}

template <typename T, class V>
int run_gmres(ht_ctx* c, double dt, const V& w, const T* b, int slot, double tol, int max_iter, int* iters) {
    const long long n = c->grid.nn;
    const int G = vec_grid(c);
    const int S = c->part_stride;
    const int m = c->opts.restart > 1 ? c->opts.restart : 200;
    HT_TRY(ensure_basis(c, m, sizeof(T) == 4));
    T* Vb = gm_basis<T>(c);
    const long long ldv = n;
    Scal* sc = c->scal + slot;
    Gmres* gm = c->gm + (slot == 0 ? 0 : 1);
    const double tol2 = tol * tol;
    int total = 0;
    for (int cycle = 0;; ++cycle) {
        HT_TRY(apply_T<T>(c, HT_TEMP, dt, w.x, w.q, nullptr, nullptr, nullptr));
        gm_init_kernel<T><<<G, kVecThreads, 0, c->stream>>>(n, b, w.q, Vb, c->part, S); ++c->n_launch;
        HT_CUDA(c, cudaMemsetAsync(sc, 0, sizeof(Scal), c->stream));
        gm_scalar_kernel<<<1, 256, 0, c->stream>>>(GM_INIT, 0, c->part, S, G, sc, gm, tol2, max_iter, m); ++c->n_launch;
        HT_CUDA(c, cudaGetLastError());
        HT_TRY(sync_scal(c, slot));
        Scal st = c->scal_host[slot];
        if (st.bb == 0.0) {
            fill_kernel<T><<<G, kVecThreads, 0, c->stream>>>(n, w.x, T(0)); ++c->n_launch;
            break;
        }
        if (st.conv || st.status != ST_OK) break;
        if (total >= max_iter) break;
        const int mm = std::min(m, max_iter - total);
        int check = 8;
        int next_check = check - 1;
        for (int k = 0; k < mm; ++k) {
            T* vk = Vb + (size_t)k * ldv;
            T* wv = Vb + (size_t)(k + 1) * ldv;
            const dim3 dg(G, (k + 1 + kDotChunk - 1) / kDotChunk);
            gm_prep_kernel<T><<<G, kVecThreads, 0, c->stream>>>(n, vk, w.Dinv, w.ph, gm, sc); ++c->n_launch;
            HT_TRY(apply_T<T>(c, HT_TEMP, dt, w.ph, wv, nullptr, nullptr, sc));
            gm_dots_kernel<T><<<dg, kVecThreads, 0, c->stream>>>(n, Vb, ldv, k, wv, c->part, S, sc); ++c->n_launch;
            gm_hreduce_kernel<<<k + 1, 256, 0, c->stream>>>(c->part, S, G, gm, k, 1, sc); ++c->n_launch;
            gm_orth_kernel<T><<<G, kVecThreads, 0, c->stream>>>(n, Vb, ldv, k, wv, gm, 1, c->part, S, sc); ++c->n_launch;
            gm_dots_kernel<T><<<dg, kVecThreads, 0, c->stream>>>(n, Vb, ldv, k, wv, c->part, S, sc); ++c->n_launch;
            gm_hreduce_kernel<<<k + 1, 256, 0, c->stream>>>(c->part, S, G, gm, k, 2, sc); ++c->n_launch;
            gm_orth_kernel<T><<<G, kVecThreads, 0, c->stream>>>(n, Vb, ldv, k, wv, gm, 2, c->part, S, sc); ++c->n_launch;
            gm_scalar_kernel<<<1, 256, 0, c->stream>>>(GM_NORM, k, c->part, S, G, sc, gm, tol2, max_iter, mm); ++c->n_launch;
            if (k == next_check) {
                HT_CUDA(c, cudaGetLastError());
                HT_TRY(sync_scal(c, slot));
                if (c->scal_host[slot].done) break;
                if (check < 32) check *= 2;
                next_check = k + check;
            }
        }
        gm_scalar_kernel<<<1, 256, 0, c->stream>>>(GM_SOLVE, 0, c->part, S, G, sc, gm, tol2, max_iter, mm); ++c->n_launch;
        gm_update_kernel<T><<<G, kVecThreads, 0, c->stream>>>(n, Vb, ldv, gm, sc, w.Dinv, w.x); ++c->n_launch;
        HT_CUDA(c, cudaGetLastError());
        HT_TRY(sync_scal(c, slot));
        st = c->scal_host[slot];
        total += st.kdone;
        if (st.status == ST_NAN) break;
        if (total >= max_iter) break;
        // the next cycle recomputes the true residual and tests convergence
    }
    *iters = total;
    return HT_OK;
}


constexpr double kChebRatio = 30.0;

// largest eigenvalue of D^-1 A (head operator) by power iteration, cached per dt
int cheb_lambda_max(ht_ctx* c, double dt, double* lmax) {
    if (c->cheb_dt[HT_HEAD] == dt && c->cheb_lmax[HT_HEAD] > 0) {
        *lmax = c->cheb_lmax[HT_HEAD];
        return HT_OK;
    }
    const long long n = c->grid.nn;
    const int G = vec_grid(c);
    const int S = c->part_stride;
    double* v = c->rh;
    double* w = c->s;
    seed_kernel<<<G, kVecThreads, 0, c->stream>>>(n, v); ++c->n_launch;
    double norm = 1.0, lam = 0.0;
    for (int it = 0; it < 50; ++it) {
        HT_TRY(launch_apply64(c, HT_HEAD, dt, v, w, nullptr, nullptr, nullptr));
        power_kernel<<<G, kVecThreads, 0, c->stream>>>(n, w, c->D, v, 1.0 / norm, c->part, S); ++c->n_launch;
        scalar_kernel<<<1, 256, 0, c->stream>>>(SC_NORMS, c->part, S, G, c->scal + 3, 0.0, 0); ++c->n_launch;
        HT_CUDA(c, cudaGetLastError());
        HT_TRY(sync_scal(c, 3));
        // v now holds D^-1 A v_prev / |v_prev|: its norm estimates lambda_max
        const double nv = sqrt(c->scal_host[3].rr);
        if (it > 0) lam = nv;
        norm = nv > 0 ? nv : 1.0;
    }
    // power iteration approaches lambda_max from below; the margin keeps the
    // top of the spectrum inside the Chebyshev interval
    *lmax = 1.2 * lam;
    c->cheb_lmax[HT_HEAD] = *lmax;
    c->cheb_dt[HT_HEAD] = dt;
    return HT_OK;
}

template <typename T, class V>
int cheb_apply(ht_ctx* c, double dt, const V& w, const T* r, T* z, T* d, T* tmp, double lmax, const Scal* sc) {
    const long long n = c->grid.nn;
    const int G = vec_grid(c);
    const int k = c->opts.cheb_degree > 0 ? c->opts.cheb_degree : 4;
    const double b = lmax, a = lmax / kChebRatio;
    const double theta = 0.5 * (b + a), delta = 0.5 * (b - a), sigma = theta / delta;
    cheb_init_kernel<T><<<G, kVecThreads, 0, c->stream>>>(n, r, w.Dinv, d, z, (T)(1.0 / theta), sc); ++c->n_launch;
    double rho_prev = 1.0 / sigma;
    for (int j = 1; j < k; ++j) {
        const double rho = 1.0 / (2.0 * sigma - rho_prev);
        HT_TRY(apply_T<T>(c, HT_HEAD, dt, z, tmp, nullptr, nullptr, sc));
        cheb_step_kernel<T><<<G, kVecThreads, 0, c->stream>>>(n, r, tmp, w.Dinv, d, z, (T)(rho * rho_prev),
                                                              (T)(2.0 * rho / delta), sc); ++c->n_launch;
        rho_prev = rho;
    }
    HT_CUDA(c, cudaGetLastError());
    return HT_OK;
}

// CG preconditioned by the Chebyshev-Jacobi polynomial.  beta takes the
// flexible (Polak-Ribiere) form -alpha z_new.q / r_old.z_old, equal to the
// usual r_new.z_new / r_old.z_old in exact arithmetic but robust to the
// rounding of a degree-k polynomial applied in FP32.
template <typename T, class V>
int run_cg_cheb(ht_ctx* c, double dt, const V& w, T* z, T* d, T* tmp, const T* b, int slot, double tol,
                int max_iter, int* iters) {
    const long long n = c->grid.nn;
    const int G = vec_grid(c);
    const int S = c->part_stride;
    Scal* sc = c->scal + slot;
    double lmax = 0;
    HT_TRY(cheb_lambda_max(c, dt, &lmax));
    int np = 0;
    HT_TRY(apply_T<T>(c, HT_HEAD, dt, w.x, w.q, nullptr, nullptr, nullptr));
    cgz_init_kernel<T><<<G, kVecThreads, 0, c->stream>>>(n, b, w.q, w.r, c->part, S); ++c->n_launch;
    HT_CUDA(c, cudaMemsetAsync(sc, 0, sizeof(Scal), c->stream));
    HT_TRY((cheb_apply<T, V>(c, dt, w, w.r, z, d, tmp, lmax, nullptr)));
    cgz_dot_kernel<T><<<G, kVecThreads, 0, c->stream>>>(n, w.r, z, (const T*)nullptr, c->part, S, 0, sc); ++c->n_launch;
    HT_TRY(scalar(c, SC_CG_INIT, G, slot, tol, max_iter));
    copy_kernel<T><<<G, kVecThreads, 0, c->stream>>>(n, z, w.p); ++c->n_launch;
    HT_TRY(sync_scal(c, slot));
    if (c->scal_host[slot].bb == 0.0) {
        fill_kernel<T><<<G, kVecThreads, 0, c->stream>>>(n, w.x, T(0)); ++c->n_launch;
        *iters = 0;
        return HT_OK;
    }
    int chunk = c->opts.check_every > 0 ? c->opts.check_every : 8;
    while (!c->scal_host[slot].done) {
        for (int it = 0; it < chunk; ++it) {
            HT_TRY(apply_T<T>(c, HT_HEAD, dt, w.p, w.q, c->part, &np, sc));
            HT_TRY(scalar(c, SC_CG_ALPHA, np, slot, tol, max_iter));
            cgz_update_kernel<T><<<G, kVecThreads, 0, c->stream>>>(n, w.x, w.r, w.p, w.q, sc, c->part, S); ++c->n_launch;
            HT_TRY((cheb_apply<T, V>(c, dt, w, w.r, z, d, tmp, lmax, sc)));
            cgz_dot_kernel<T><<<G, kVecThreads, 0, c->stream>>>(n, w.r, z, w.q, c->part, S, 1, sc); ++c->n_launch;
            HT_TRY(scalar(c, SC_FCG_BETA, G, slot, tol, max_iter));
            cgz_pupdate_kernel<T><<<G, kVecThreads, 0, c->stream>>>(n, z, w.p, sc); ++c->n_launch;
        }
        HT_CUDA(c, cudaGetLastError());
        HT_TRY(sync_scal(c, slot));
        if (chunk < 32) chunk *= 2;
    }
    *iters = c->scal_host[slot].iters;
    return HT_OK;
}

__global__ void inv32_kernel(long long n, const float* __restrict__ D, float* __restrict__ Dinv32) {
    GRID_LOOP(i, n) Dinv32[i] = 1.0f / D[i];
}

int prepare_diag(ht_ctx* c, int field, double dt) {
    // The FP32 inner solves of the mixed form use only the FP32 inverse
    // diagonal, so it is computed in FP32; the Chebyshev bounds of the head
    // CG come from the FP64 diagonal.
    if (c->opts.precision == HT_MIXED && !(field == HT_HEAD && c->opts.precond == HT_PREC_CHEBYSHEV)) {
        HT_TRY(launch_diag32(c, field, dt, c->z32));
        inv32_kernel<<<vec_grid(c), kVecThreads, 0, c->stream>>>(c->grid.nn, c->z32, c->D32); ++c->n_launch;
        HT_CUDA(c, cudaGetLastError());
        return HT_OK;
    }
    HT_TRY(launch_diag(c, field, dt, c->z));
    inv_kernel<<<vec_grid(c), kVecThreads, 0, c->stream>>>(c->grid.nn, c->z, c->D, c->D32); ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    return HT_OK;
}

int status_to_rc(ht_ctx* c, const Scal& s, double tol, const char* what) {
    if (s.status == ST_NAN) return fail(c, HT_EINVAL, "%s: non-finite residual", what);
    if (s.status == ST_BREAKDOWN) return fail(c, HT_EBREAKDOWN, "%s: Krylov breakdown", what);
    if (s.bb > 0 && s.rr > tol * tol * s.bb)
        return fail(c, HT_ENOCONV, "%s: no convergence in %d iterations (rel. residual %.3e)", what,
                    s.iters, sqrt(s.rr / s.bb));
    return HT_OK;
}

int solve_field(ht_ctx* c, int field, double dt, double* x, const double* b, int* iters, int* outer,
                double* res) {
    const double tol = c->opts.tol;
    const int max_iter = c->opts.max_iter;
    const char* what = field == HT_HEAD ? "head solve" : "heat solve";
    // the FP32-operator residual of the initial guess, when a guess gate has
    // formed it already (consumed here; it only lets the mixed form skip
    // forming that residual again)
    const double known_fast = c->guess_fast[field];
    c->guess_fast[field] = -1.0;
    HT_TRY(prepare_diag(c, field, dt));
    *iters = 0;
    *outer = 0;
    if (c->opts.precision == HT_FP64) {
        Vecs64 w{x, c->r, c->p, c->q, c->D, c->rh, c->v, c->s, c->tv, c->ph, c->sh};
        int total = 0;
        // The Krylov loops stop on their recursively updated residual; the
        // true FP64 residual decides, and a pass that stopped short of it
        // restarts from the current iterate.
        for (int pass = 0; pass < 4; ++pass) {
            int it = 0;
            if (field == HT_HEAD && c->opts.precond == HT_PREC_CHEBYSHEV)
                HT_TRY((run_cg_cheb<double, Vecs64>(c, dt, w, c->z, c->z2, c->v, b, 0, tol, max_iter - total, &it)));
            else if (field == HT_HEAD) HT_TRY((run_cg<double, Vecs64>(c, dt, w, b, 0, tol, max_iter - total, &it)));
            else if (c->opts.krylov == HT_KRYLOV_GMRES)
                HT_TRY((run_gmres<double, Vecs64>(c, dt, w, b, 0, tol, max_iter - total, &it)));
            else HT_TRY((run_bicgstab<double, Vecs64>(c, dt, w, b, 0, tol, max_iter - total, &it)));
            total += it;
            *outer = pass + 1;
            HT_TRY(true_residual(c, field, dt, x, b, res));
            const Scal s = c->scal_host[0];
            if (s.status == ST_NAN || !isfinite(*res)) return fail(c, HT_EINVAL, "%s: non-finite residual", what);
            if (*res <= tol) break;
            if (total >= max_iter || pass == 3) {
                *iters = total;
                if (s.status == ST_BREAKDOWN) return fail(c, HT_EBREAKDOWN, "%s: Krylov breakdown", what);
                return fail(c, HT_ENOCONV, "%s: no convergence in %d iterations (rel. residual %.3e)", what,
                            total, *res);
            }
        }
        *iters = total;
        return HT_OK;
    }
    // mixed precision: FP64 defect correction around FP32 inner Krylov
    const long long n = c->grid.nn;
    const int G = vec_grid(c);
    const int S = c->part_stride;
    if (field == HT_TEMP) {
        // the FP32 heat operator forms its velocity from an FP32 copy of h^{n+1}
        to_f32_kernel<<<G, kVecThreads, 0, c->stream>>>(n, c->h, c->h32); ++c->n_launch;
        HT_CUDA(c, cudaGetLastError());
    }
    const double inner_head = c->opts.inner_tol > 0 ? c->opts.inner_tol : 1e-4;
    const double inner_tol = field == HT_TEMP && c->opts.inner_tol_heat > 0 ? c->opts.inner_tol_heat : inner_head;
    const int max_outer = c->opts.max_outer > 0 ? c->opts.max_outer : 30;
    Vecs32 w{c->d32, c->r32, c->p32, c->q32, c->D32, c->rh32, c->v32, c->s32, c->t32, c->ph32, c->sh32};
    int total = 0;
    // The first outer residual only seeds the first correction, so it is
    // formed with the FP32 operator while that is accurate enough: its
    // rounding noise is about 1e-7 of ||b||, and the correction it seeds must
    // not solve for noise above the inner tolerance.  A guess whose residual
    // is below 1e-6 / inner_tol of ||b|| (a good previous or extrapolated
    // field) has its first residual formed again with the accurate operator.
    // Every later residual, and any residual that ends the loop, is formed
    // with the accurate (float-float or FP64) one.
    auto outer_residual = [&](bool fast, int* np) -> int {
        *np = G;
        if (fast) {
            to_f32_kernel<<<G, kVecThreads, 0, c->stream>>>(n, x, c->x32); ++c->n_launch;
            HT_TRY(launch_apply32(c, field, (float)dt, c->x32, c->q32, nullptr, nullptr, nullptr));
            Grid gf = c->grid;
            gf.dmask = c->dmask[field];
            resid32_kernel<<<G, kVecThreads, 0, c->stream>>>(gf, n, b, c->q32, x, c->r32, c->part, S); ++c->n_launch;
            HT_CUDA(c, cudaGetLastError());
        } else if (c->opts.outer_fp64 || (field == HT_TEMP && !heat_fused_ok(c))) {
            HT_TRY(launch_apply64(c, field, dt, x, c->q, nullptr, nullptr, nullptr));
            resid_kernel<<<G, kVecThreads, 0, c->stream>>>(n, b, c->q, nullptr, c->r32, c->part, S); ++c->n_launch;
            HT_CUDA(c, cudaGetLastError());
        } else {
            HT_TRY(launch_resid_df(c, field, dt, x, b, c->r32, c->part, np));
        }
        scalar_kernel<<<1, 256, 0, c->stream>>>(SC_NORMS, c->part, S, *np, c->scal + 2, 0.0, 0); ++c->n_launch;
        HT_CUDA(c, cudaGetLastError());
        return sync_scal(c, 2);
    };
    const double floor_rel = 1e-6 / inner_tol;
    for (int k = 0; k <= max_outer; ++k) {
        int np = G;
        const bool fast = k == 0 && !(known_fast >= 0 && known_fast < floor_rel);
        HT_TRY(outer_residual(fast, &np));
        if (fast) {
            const Scal f = c->scal_host[2];
            if (f.rr <= tol * tol * f.bb || f.rr < floor_rel * floor_rel * f.bb)
                HT_TRY(outer_residual(false, &np));   // confirm convergence, or seed accurately
        }
        const Scal s = c->scal_host[2];
        if (!isfinite(s.rr)) return fail(c, HT_EINVAL, "%s: non-finite residual", what);
        *res = s.bb > 0 ? sqrt(s.rr / s.bb) : 0.0;
        *outer = k;
        if (s.rr <= tol * tol * s.bb) break;
        if (k == max_outer || total >= max_iter)
            return fail(c, HT_ENOCONV, "%s: mixed precision stalled at rel. residual %.3e after %d outer passes",
                        what, *res, k);
        fill_kernel<float><<<G, kVecThreads, 0, c->stream>>>(n, c->d32, 0.0f); ++c->n_launch;
        HT_CUDA(c, cudaGetLastError());
        // the inner solve need not reduce the residual further than the
        // outer tolerance requires (half of it, for margin)
        const double need = s.rr > 0 ? 0.5 * tol * sqrt(s.bb / s.rr) : 1.0;
        const double itol = std::max(inner_tol, std::min(need, 0.5));
        int it = 0;
        c->cur_hint = k < 8 ? c->iter_hint[field][k] : 0;
        if (field == HT_HEAD && c->opts.precond == HT_PREC_CHEBYSHEV)
            HT_TRY((run_cg_cheb<float, Vecs32>(c, dt, w, c->z32, c->zz32, c->v32, c->r32, 1, itol,
                                               max_iter - total, &it)));
        else if (field == HT_HEAD)
            HT_TRY((run_cg<float, Vecs32>(c, dt, w, c->r32, 1, itol, max_iter - total, &it)));
        else if (c->opts.krylov == HT_KRYLOV_GMRES)
            HT_TRY((run_gmres<float, Vecs32>(c, dt, w, c->r32, 1, itol, max_iter - total, &it)));
        else
            HT_TRY((run_bicgstab<float, Vecs32>(c, dt, w, c->r32, 1, itol, max_iter - total, &it)));
        c->cur_hint = 0;
        if (k < 8) c->iter_hint[field][k] = it;
        total += it;
        if (c->scal_host[1].status == ST_NAN)
            return fail(c, HT_EINVAL, "%s: FP32 inner solve produced non-finite values", what);
        add_f32_kernel<<<G, kVecThreads, 0, c->stream>>>(n, x, c->d32); ++c->n_launch;
        HT_CUDA(c, cudaGetLastError());
    }
    *iters = total;
    return HT_OK;
}

}  // namespace

int true_residual(ht_ctx* c, int field, double dt, const double* x, const double* b, double* rel) {
    const int G = vec_grid(c);
    HT_TRY(launch_apply64(c, field, dt, x, c->q, nullptr, nullptr, nullptr));
    resid_kernel<<<G, kVecThreads, 0, c->stream>>>(c->grid.nn, b, c->q, nullptr, nullptr, c->part,
                                                    c->part_stride); ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    scalar_kernel<<<1, 256, 0, c->stream>>>(SC_NORMS, c->part, c->part_stride, G, c->scal + 3, 0.0, 0); ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    HT_TRY(sync_scal(c, 3));
    const Scal s = c->scal_host[3];
    *rel = s.bb > 0 ? sqrt(s.rr / s.bb) : sqrt(s.rr);
    return HT_OK;
}

int fast_residual(ht_ctx* c, int field, double dt, const double* x, const double* b, double* rel) {
    const long long n = c->grid.nn;
    const int G = vec_grid(c), S = c->part_stride;
    if (field == HT_TEMP) {   // the FP32 heat operator forms its velocity from the FP32 head
        to_f32_kernel<<<G, kVecThreads, 0, c->stream>>>(n, c->h, c->h32); ++c->n_launch;
    }
    to_f32_kernel<<<G, kVecThreads, 0, c->stream>>>(n, x, c->x32); ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    HT_TRY(launch_apply32(c, field, (float)dt, c->x32, c->q32, nullptr, nullptr, nullptr));
    Grid gf = c->grid;
    gf.dmask = c->dmask[field];
    resid32_kernel<<<G, kVecThreads, 0, c->stream>>>(gf, n, b, c->q32, x, c->r32, c->part, S); ++c->n_launch;
    scalar_kernel<<<1, 256, 0, c->stream>>>(SC_NORMS, c->part, S, G, c->scal + 3, 0.0, 0); ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    HT_TRY(sync_scal(c, 3));
    const Scal s = c->scal_host[3];
    *rel = s.bb > 0 ? sqrt(s.rr / s.bb) : sqrt(s.rr);
    return HT_OK;
}

// r = b - q, partial sums of r.r and b.b (slots 0 and 1); *n_part entries
int launch_resid64(ht_ctx* c, const double* b, const double* q, double* part, int* n_part) {
    const int G = vec_grid(c);
    resid_kernel<<<G, kVecThreads, 0, c->stream>>>(c->grid.nn, b, q, nullptr, nullptr, part, c->part_stride);
    ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    *n_part = G;
    return HT_OK;
}

// reduce the r.r / b.b partial sums into c->scal[slot] (rr, bb)
int launch_norms(ht_ctx* c, int n_part, int slot) {
    scalar_kernel<<<1, 256, 0, c->stream>>>(SC_NORMS, c->part, c->part_stride, n_part, c->scal + slot, 0.0, 0);
    ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    return HT_OK;
}

int set_dirichlet_values(ht_ctx* c, int field, double* x) {
    Grid g = c->grid;
    g.dmask = c->dmask[field];
    if (field == HT_TEMP) HT_TRY(dint_scatter(c, x, c->g[HT_TEMP]));   // pile surfaces off the faces
    if (!g.dmask) return HT_OK;
    dirichlet_kernel<<<vec_grid(c), kVecThreads, 0, c->stream>>>(g, c->g[field], x); ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    return HT_OK;
}

// z = w0 y0 + w1 y1 + w2 y2 over the first `deg` + 1 terms, then y2 = y0
// (the buffer of the oldest past field takes the current one)
static __global__ void extrap_kernel(long long n, const double* __restrict__ y0, const double* __restrict__ y1,
                                     double* __restrict__ y2, int deg, double w0, double w1, double w2,
                                     double* __restrict__ z) {
    GRID_LOOP(i, n) {
        const double a = y0[i];
        double v = w0 * a;
        if (deg >= 1) v += w1 * y1[i];
        if (deg >= 2) v += w2 * y2[i];
        if (z) z[i] = v;
        y2[i] = a;
    }
}

int guess_extrapolate(ht_ctx* c, int field, double t1, double* z, int* deg) {
    *deg = 0;
    const size_t n = (size_t)c->grid.nn;
    for (double*& p : c->gpast[field])
        if (!p && cudaMalloc(&p, n * sizeof(double)) != cudaSuccess) {
            c->ghist = 0;
            return fail(c, HT_ENOMEM, "extrapolated guess: allocation failed");
        }
    // Lagrange weights at t1 through (t^n, y0), (gtime[0], y1), (gtime[1], y2);
    // the times must be distinct and decreasing, else fewer points are used
    const double tn = c->t, ta = c->gtime[0], tb = c->gtime[1];
    int d = c->ghist;
    if (d >= 2 && !(ta > tb)) d = 1;
    if (d >= 1 && !(tn > ta)) d = 0;
    double w[3] = {1.0, 0.0, 0.0};
    if (d == 1) {
        w[0] = (t1 - ta) / (tn - ta);
        w[1] = (t1 - tn) / (ta - tn);
    } else if (d == 2) {
        w[0] = (t1 - ta) * (t1 - tb) / ((tn - ta) * (tn - tb));
        w[1] = (t1 - tn) * (t1 - tb) / ((ta - tn) * (ta - tb));
        w[2] = (t1 - tn) * (t1 - ta) / ((tb - tn) * (tb - ta));
    }
    double* y0 = field == HT_HEAD ? c->h : c->T;
    extrap_kernel<<<vec_grid(c), kVecThreads, 0, c->stream>>>((long long)n, y0, c->gpast[field][0], c->gpast[field][1],
                                                              d, w[0], w[1], w[2], d > 0 ? z : nullptr);
    ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    std::swap(c->gpast[field][0], c->gpast[field][1]);   // the newest past field is y0
    if (d > 0) HT_TRY(set_dirichlet_values(c, field, z));
    *deg = d;
    return HT_OK;
}

void guess_commit(ht_ctx* c, double t_prev) {
    c->gtime[1] = c->gtime[0];
    c->gtime[0] = t_prev;
    c->ghist = std::min(c->ghist + 1, 2);
}

void guess_free(ht_ctx* c) {
    for (auto& f : c->gpast)
        for (double*& p : f) {
            if (p) cudaFree(p);
            p = nullptr;
        }
    c->ghist = 0;
}

int solve_head(ht_ctx* c, double dt, double* x, const double* b, int* iters, int* outer, double* res) {
    return solve_field(c, HT_HEAD, dt, x, b, iters, outer, res);
}

int solve_heat(ht_ctx* c, double dt, double* x, const double* b, int* iters, int* outer, double* res) {
    return solve_field(c, HT_TEMP, dt, x, b, iters, outer, res);
}


// ---- pieces of the head solve used by the batched step (ht_batch.cu) ----------------
int batch_prepare_diag(ht_ctx* c, double dt) { return prepare_diag(c, HT_HEAD, dt); }

// FP64 residual r = b - A x of the head system; r32 = (float) r; convergence test
int batch_outer_residual(ht_ctx* c, double dt, double tol, int* converged, double* res) {
    const int G = vec_grid(c);
    HT_TRY(launch_apply64(c, HT_HEAD, dt, c->x, c->q, nullptr, nullptr, nullptr));
    resid_kernel<<<G, kVecThreads, 0, c->stream>>>(c->grid.nn, c->b, c->q, nullptr, c->r32, c->part, c->part_stride); ++c->n_launch;
    scalar_kernel<<<1, 256, 0, c->stream>>>(SC_NORMS, c->part, c->part_stride, G, c->scal + 2, 0.0, 0); ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    HT_TRY(sync_scal(c, 2));
    const Scal s = c->scal_host[2];
    if (!isfinite(s.rr)) return fail(c, HT_EINVAL, "head solve: non-finite residual");
    *res = s.bb > 0 ? sqrt(s.rr / s.bb) : 0.0;
    *converged = (s.rr <= tol * tol * s.bb) ? 1 : 0;
    return HT_OK;
}

// the same residual without the host wait: the norms land in scal_host[2]
// once the stream reaches the copy (batch_outer_residual_read after a sync)
int batch_outer_residual_enqueue(ht_ctx* c, double dt) {
    const int G = vec_grid(c);
    HT_TRY(launch_apply64(c, HT_HEAD, dt, c->x, c->q, nullptr, nullptr, nullptr));
    resid_kernel<<<G, kVecThreads, 0, c->stream>>>(c->grid.nn, c->b, c->q, nullptr, c->r32, c->part, c->part_stride); ++c->n_launch;
    scalar_kernel<<<1, 256, 0, c->stream>>>(SC_NORMS, c->part, c->part_stride, G, c->scal + 2, 0.0, 0); ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    HT_CUDA(c, cudaMemcpyAsync(c->scal_host + 2, c->scal + 2, sizeof(Scal), cudaMemcpyDeviceToHost, c->stream));
    return HT_OK;
}

int batch_outer_residual_read(ht_ctx* c, double tol, int* converged, double* res) {
    const Scal s = c->scal_host[2];
    if (!isfinite(s.rr)) return fail(c, HT_EINVAL, "head solve: non-finite residual");
    *res = s.bb > 0 ? sqrt(s.rr / s.bb) : 0.0;
    *converged = (s.rr <= tol * tol * s.bb) ? 1 : 0;
    return HT_OK;
}

// x += d and the inner scalars to scal_host[1], without the host wait (the
// caller checks scal_host[1].status after a sync)
int batch_outer_update_enqueue(ht_ctx* c) {
    HT_CUDA(c, cudaMemcpyAsync(c->scal_host + 1, c->scal + 1, sizeof(Scal), cudaMemcpyDeviceToHost, c->stream));
    add_f32_kernel<<<vec_grid(c), kVecThreads, 0, c->stream>>>(c->grid.nn, c->x, c->d32); ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    return HT_OK;
}

// start the inner FP32 CG on A32 d = r32 (d = 0); scalars in slot 1
int batch_inner_init(ht_ctx* c, double dt, double inner_tol, int max_iter) {
    const long long n = c->grid.nn;
    const int G = vec_grid(c);
    fill_kernel<float><<<G, kVecThreads, 0, c->stream>>>(n, c->d32, 0.0f); ++c->n_launch;
    HT_TRY(launch_apply32(c, HT_HEAD, (float)dt, c->d32, c->q32, nullptr, nullptr, nullptr));
    cg_init_kernel<float><<<G, kVecThreads, 0, c->stream>>>(n, c->r32, c->q32, c->D32, c->r32, c->p32, c->part,
                                                            c->part_stride); ++c->n_launch;
    HT_CUDA(c, cudaMemsetAsync(c->scal + 1, 0, sizeof(Scal), c->stream));
    scalar_kernel<<<1, 256, 0, c->stream>>>(SC_CG_INIT, c->part, c->part_stride, G, c->scal + 1,
                                            inner_tol * inner_tol, max_iter); ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    return HT_OK;
}

// x += d after the batched inner solve; reads back the inner scalars
int batch_outer_update(ht_ctx* c) {
    HT_TRY(sync_scal(c, 1));
    if (c->scal_host[1].status == ST_NAN) return fail(c, HT_EINVAL, "head solve: FP32 inner solve produced non-finite values");
    add_f32_kernel<<<vec_grid(c), kVecThreads, 0, c->stream>>>(c->grid.nn, c->x, c->d32); ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    return HT_OK;
}

}  // namespace ht

