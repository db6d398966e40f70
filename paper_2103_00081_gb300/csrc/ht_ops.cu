// Matrix-free operator kernels of the head and heat systems on a structured
// box of Q1 / Q2 hexahedra (Section 2, Eq. 3 and Eq. 4 in head / energy form).
//
// Tiling ("owner computes", deterministic, no atomics):
//   * a CTA owns a TX x TY column of nodes (TX = P*(CXM-1), TY = P*(CYM-1))
//     and a chunk of node planes in z;
//   * it marches upward through the cell layers that touch its planes; in
//     each layer one thread computes one cell (the CXM x CYM cells touching
//     the owned columns, including a one-cell halo on the low side) and
//     writes the element result to shared memory;
//   * each owned node then sums the contributions of its (up to 4) cells of
//     the layer in a fixed order, adds the carry of the plane it shares with
//     the layer below and emits the finished planes.
// Every node value is therefore produced by exactly one thread, in a fixed
// summation order, and the kernels are bitwise reproducible.
//
// Cell work:
//   * head operator alpha M_e + beta_c K_e (beta_c = dt K_c): sum
//     factorisation in the 1D generalised eigenbasis of (k, m) ("fast
//     diagonalisation"): three 1D transforms, one scaling per mode, three
//     transposed transforms;
//   * heat operator c_T M_e + dt lambda K_e + dt C_e(q): sum-factorised
//     Gauss quadrature of the weak form of Eq. 4 with the Darcy flux
//     q = -K_c grad h^{n+1} at the Gauss points.
#include <cuda_runtime.h>
#include <stdio.h>

#include <mutex>
#include <type_traits>

#include "ht_device.cuh"
#include "ht_internal.cuh"

namespace ht {

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool on_dir(const Grid& g, int i, int j, int k) {
    const int m = g.dmask;
    return ((m & 1) && i == 0) || ((m & 2) && i == g.Nx - 1) || ((m & 4) && j == 0) ||
           ((m & 8) && j == g.Ny - 1) || ((m & 16) && k == 0) || ((m & 32) && k == g.Nz - 1);
}

__device__ __forceinline__ bool cell_touches_dir(const Grid& g, int cx, int cy, int cz) {
    const int m = g.dmask;
    return ((m & 1) && cx == 0) || ((m & 2) && cx == g.ncx - 1) || ((m & 4) && cy == 0) ||
           ((m & 8) && cy == g.ncy - 1) || ((m & 16) && cz == 0) || ((m & 32) && cz == g.ncz - 1);
}

__device__ __forceinline__ long long nidx(const Grid& g, int i, int j, int k) {
    return (long long)i + (long long)g.Nx * ((long long)j + (long long)g.Ny * k);
}

template <typename T>
__device__ __forceinline__ T ldro(const T* p) { return __ldg(p); }

// ---------------------------------------------------------------------------
// Float-float arithmetic (emulated FP64 on the FP32 pipes, which GB300 runs
// at 64x its FP64 rate).  Error-free transformations: TwoSum (Knuth, TAOCP
// vol. 2, 4.2.2), FastTwoSum for |a| >= |b| (Dekker 1971) and TwoProduct
// with a fused multiply-add; the compound addition adds the low parts
// without a second TwoSum (Dekker's addition), so its error is of order
// 2^-46 (|a| + |b|) and the product's 2^-46 |ab|.  The _rn intrinsics keep
// the compiler from contracting the steps into other fused operations.
// ---------------------------------------------------------------------------
__device__ __forceinline__ df64 df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df64(s, e);
}
__device__ __forceinline__ df64 df_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return df64(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
    const df64 s = df_two_sum(a.hi, b.hi);
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}
__device__ __forceinline__ df64& operator+=(df64& a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64& operator*=(df64& a, df64 b) { return a = a * b; }
using ::fma;   // keep the float and double overloads visible beside the float-float one
__device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c) { return a * b + c; }
__device__ __forceinline__ df64 df_from(double d) {
    const float hi = __double2float_rn(d);
    return df64(hi, __double2float_rn(d - (double)hi));
}
__device__ __forceinline__ double df_to(df64 a) { return (double)a.hi + (double)a.lo; }

// read-only load of any of the element types
template <typename T>
__device__ __forceinline__ T ldg_any(const T* p) { return __ldg(p); }
template <>
__device__ __forceinline__ df64 ldg_any<df64>(const df64* p) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return df64(v.x, v.y);
}

// value of storage type S in compute type T
template <typename T, typename S>
struct Cvt {
    __device__ __forceinline__ static T f(S v) { return (T)v; }
};
template <>
struct Cvt<df64, double> {
    __device__ __forceinline__ static df64 f(double v) { return df_from(v); }
};
template <typename T, typename S>
__device__ __forceinline__ T cvt(S v) { return Cvt<T, S>::f(v); }

// gather the element vector of cell (cx,cy,cz) from a nodal vector; nodes on
// Dirichlet faces read as zero when `mask` is set.
template <int P, typename T>
__device__ __forceinline__ void gather(const Grid& g, const T* __restrict__ x, int cx, int cy,
                                       int cz, bool mask, T (&u)[(P + 1) * (P + 1) * (P + 1)]) {
    constexpr int n = P + 1;
    const int i0 = P * cx, j0 = P * cy, k0 = P * cz;
    const bool chk = mask && cell_touches_dir(g, cx, cy, cz);
#pragma unroll
    for (int c = 0; c < n; ++c)
#pragma unroll
        for (int b = 0; b < n; ++b) {
            const T* row = x + nidx(g, i0, j0 + b, k0 + c);
#pragma unroll
            for (int a = 0; a < n; ++a) {
                T v = ldro(row + a);
                if (chk && on_dir(g, i0 + a, j0 + b, k0 + c)) v = T(0);
                u[a + n * (b + n * c)] = v;
            }
        }
}

// 1D transforms of an n^3 array u[c][b][a] along one axis with matrix M
// (TR: use M^T).  out[i] = sum_a M[i][a] in[a].
template <int n, int AX, bool TR, typename T>
__device__ __forceinline__ void sweep(T (&u)[n * n * n], const T (&M)[3][3]) {
    constexpr int st = AX == 0 ? 1 : (AX == 1 ? n : n * n);
#pragma unroll
    for (int l = 0; l < n * n; ++l) {
        // base index of the line: the two other coordinates
        int base;
        if (AX == 0) base = l * n;
        else if (AX == 1) base = (l % n) + (l / n) * n * n;
        else base = l;
        T in[n], out[n];
#pragma unroll
        for (int a = 0; a < n; ++a) in[a] = u[base + a * st];
#pragma unroll
        for (int i = 0; i < n; ++i) {
            T s = T(0);
#pragma unroll
            for (int a = 0; a < n; ++a) s = fma(TR ? M[a][i] : M[i][a], in[a], s);
            out[i] = s;
        }
#pragma unroll
        for (int i = 0; i < n; ++i) u[base + i * st] = out[i];
    }
}

// ---------------------------------------------------------------------------
// Operators (cell computation + node emission)
// ---------------------------------------------------------------------------
// Per-cell geometry of a graded mesh (Fig. 10b: tensor-product cell widths):
// geo[k * nc + c] = volume, 1/hx, 1/hy, 1/hz of cell c in storage type S;
// null on a uniform mesh, whose element constants carry the cell size.  On a
// graded mesh the element constants are those of the unit cube and each
// cell scales them: the volume scales mass and Gauss weights, 1/h_d each
// derivative along d (for the fast diagonalisation: G = sqrt(h) G_1 per
// axis, so the cell matrix is vol (G_1^T)^3 diag(alpha + beta sum_d
// Lam_1,d / h_d^2) G_1^3).
template <typename T, typename S>
struct CellGeo {
    const S* geo;
    long long gnc;
    __device__ __forceinline__ void geom(long long c, T& vol, T (&ih)[3]) const {
        vol = cvt<T>(ldro(geo + c));
#pragma unroll
        for (int d = 0; d < 3; ++d) ih[d] = cvt<T>(ldro(geo + (d + 1) * gnc + c));
    }
};

template <int P, typename T, int MODE, typename S = T>
struct HeadOp : CellGeo<T, S> {
    static constexpr int n = P + 1, NL = n * n * n;
    static constexpr bool kPlanes = false;
    const T* x;        // APPLY: input; RHS: u_old
    const double* gD;  // RHS: Dirichlet values
    const double* F;   // RHS: loads
    T* y;
    const S* K;        // per cell, in storage type S (converted to T on load)
    T alpha, dt;
    Elem<T> e;

    __device__ __forceinline__ void cell(const Grid& g, int cx, int cy, int cz, long long c,
                                         T (&res)[NL]) const {
        const T beta = dt * cvt<T>(ldro(K + c));
        if (MODE == MODE_DIAG) {
            if (this->geo) {
                T vol, ih[3];
                this->geom(c, vol, ih);
                const T i0 = ih[0] * ih[0], i1 = ih[1] * ih[1], i2 = ih[2] * ih[2];
#pragma unroll
                for (int cc = 0; cc < n; ++cc)
#pragma unroll
                    for (int b = 0; b < n; ++b)
#pragma unroll
                        for (int a = 0; a < n; ++a) {
                            const T dm = e.dm1[a] * e.dm1[b] * e.dm1[cc];
                            const T dk = e.dk1[a] * i0 * e.dm1[b] * e.dm1[cc] + e.dm1[a] * e.dk1[b] * i1 * e.dm1[cc] +
                                         e.dm1[a] * e.dm1[b] * e.dk1[cc] * i2;
                            res[a + n * (b + n * cc)] = vol * fma(beta, dk, alpha * dm);
                        }
                return;
            }
#pragma unroll
            for (int l = 0; l < NL; ++l) res[l] = fma(beta, e.dK[l], alpha * e.dM[l]);
            return;
        }
        if (MODE == MODE_APPLY) {
            gather<P, T>(g, x, cx, cy, cz, true, res);
            fdm(res, beta, c);
            return;
        } else if (!cell_touches_dir(g, cx, cy, cz)) {
            rhs_interior(g, cx, cy, cz, res);
            return;
        } else {  // RHS: alpha M (u_old - g_D) - beta K g_D
            T us[NL];
            const int i0 = P * cx, j0 = P * cy, k0 = P * cz;
#pragma unroll
            for (int c2 = 0; c2 < n; ++c2)
#pragma unroll
                for (int b = 0; b < n; ++b)
#pragma unroll
                    for (int a = 0; a < n; ++a) {
                        const int l = a + n * (b + n * c2);
                        const long long id = nidx(g, i0 + a, j0 + b, k0 + c2);
                        const bool d = on_dir(g, i0 + a, j0 + b, k0 + c2);
                        const T gv = d ? (T)gD[id] : T(0);
                        res[l] = x[id] - gv;
                        us[l] = gv;
                    }
            sweep<n, 0, false>(res, e.G[0]);
            sweep<n, 1, false>(res, e.G[1]);
            sweep<n, 2, false>(res, e.G[2]);
            sweep<n, 0, false>(us, e.G[0]);
            sweep<n, 1, false>(us, e.G[1]);
            sweep<n, 2, false>(us, e.G[2]);
            T vol = T(1), i2[3] = {T(1), T(1), T(1)};
            if (this->geo) {
                this->geom(c, vol, i2);
#pragma unroll
                for (int d = 0; d < 3; ++d) i2[d] = i2[d] * i2[d];
            }
#pragma unroll
            for (int c2 = 0; c2 < n; ++c2)
#pragma unroll
                for (int b = 0; b < n; ++b)
#pragma unroll
                    for (int a = 0; a < n; ++a) {
                        const int l = a + n * (b + n * c2);
                        res[l] = vol * (alpha * res[l] -
                                        beta * (e.Lam[0][a] * i2[0] + e.Lam[1][b] * i2[1] + e.Lam[2][c2] * i2[2]) *
                                            us[l]);
                    }
        }
        sweep<n, 2, true>(res, e.G[2]);
        sweep<n, 1, true>(res, e.G[1]);
        sweep<n, 0, true>(res, e.G[0]);
    }

    // RHS of a cell without Dirichlet nodes: g_D vanishes on it, so the
    // element result is alpha M u_old = alpha (G^T)^3 G^3 u_old
    __device__ __forceinline__ void rhs_interior(const Grid& g, int cx, int cy, int cz, T (&res)[NL]) const {
        gather<P, T>(g, x, cx, cy, cz, false, res);
        sweep<n, 0, false>(res, e.G[0]);
        sweep<n, 1, false>(res, e.G[1]);
        sweep<n, 2, false>(res, e.G[2]);
        T sa = alpha;
        if (this->geo) {
            T vol, ih[3];
            this->geom((long long)cx + (long long)g.ncx * ((long long)cy + (long long)g.ncy * cz), vol, ih);
            sa = alpha * vol;
        }
#pragma unroll
        for (int l = 0; l < NL; ++l) res[l] *= sa;
        sweep<n, 2, true>(res, e.G[2]);
        sweep<n, 1, true>(res, e.G[1]);
        sweep<n, 0, true>(res, e.G[0]);
    }

    // the scale of mode l of cell c: alpha + beta LS_l (uniform mesh) or
    // vol (alpha + beta sum_d Lam_d / h_d^2) (graded mesh, unit constants)
    __device__ __forceinline__ void mode_scales(long long c, const T beta, T (&sl)[NL]) const {
        if (this->geo) {
            T vol, ih[3];
            this->geom(c, vol, ih);
            const T i0 = ih[0] * ih[0], i1 = ih[1] * ih[1], i2 = ih[2] * ih[2];
#pragma unroll
            for (int cc = 0; cc < n; ++cc)
#pragma unroll
                for (int b = 0; b < n; ++b)
#pragma unroll
                    for (int a = 0; a < n; ++a)
                        sl[a + n * (b + n * cc)] =
                            vol * fma(beta, e.Lam[0][a] * i0 + e.Lam[1][b] * i1 + e.Lam[2][cc] * i2, alpha);
        } else {
#pragma unroll
            for (int l = 0; l < NL; ++l) sl[l] = fma(beta, e.LS[l], alpha);
        }
    }

    // res <- (G^T)^3 diag(alpha + beta (Lx+Ly+Lz)) G^3 res, in place
    __device__ __forceinline__ void fdm(T (&res)[NL], const T beta, long long c) const {
        sweep<n, 0, false>(res, e.G[0]);
        sweep<n, 1, false>(res, e.G[1]);
        sweep<n, 2, false>(res, e.G[2]);
        T sl[NL];
        mode_scales(c, beta, sl);
#pragma unroll
        for (int l = 0; l < NL; ++l) res[l] *= sl[l];
        sweep<n, 2, true>(res, e.G[2]);
        sweep<n, 1, true>(res, e.G[1]);
        sweep<n, 0, true>(res, e.G[0]);
    }

    // element result of the apply from the (masked) element vector u
    __device__ __forceinline__ void compute(const T (&u)[NL], long long c, T (&res)[NL]) const {
#pragma unroll
        for (int l = 0; l < NL; ++l) res[l] = u[l];
        fdm(res, dt * cvt<T>(ldro(K + c)), c);
    }

    // the same in place (u becomes A_e u), adding u^T A_e u to dot: in the
    // eigenbasis v = G^3 u the element matrix is diagonal, so the energy is
    // sum_l (alpha + beta LS_l) v_l^2 and u need not be kept
    __device__ __forceinline__ void compute_dot_inplace(T (&u)[NL], long long c, T& dot) const {
        const T beta = dt * cvt<T>(ldro(K + c));
        sweep<n, 0, false>(u, e.G[0]);
        sweep<n, 1, false>(u, e.G[1]);
        sweep<n, 2, false>(u, e.G[2]);
        T sls[NL];
        mode_scales(c, beta, sls);
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            const T sl = sls[l];
            const T v = u[l] * sl;
            dot = fma(v, u[l], dot);
            u[l] = v;
        }
        sweep<n, 2, true>(u, e.G[2]);
        sweep<n, 1, true>(u, e.G[1]);
        sweep<n, 0, true>(u, e.G[0]);
    }

    __device__ __forceinline__ void emit(const Grid& g, int i, int j, int k, T val, T& dot) const {
        const long long id = nidx(g, i, j, k);
        const bool d = on_dir(g, i, j, k);
        if (MODE == MODE_APPLY) {
            const T xv = x[id];
            const T yv = d ? xv : val;
            y[id] = yv;
            dot = fma(xv, yv, dot);
        } else if (MODE == MODE_RHS) {
            y[id] = d ? (T)gD[id] : val + dt * (T)F[id];
        } else {
            y[id] = d ? T(1) : val;
        }
    }
};

template <int P, typename T, int MODE, typename S = T>
struct HeatOp : CellGeo<T, S> {
    static constexpr int n = P + 1, NL = n * n * n, NQ = n * n * n;
    static constexpr bool kPlanes = true;   // element pass: one thread per Gauss plane
    const T* x;        // APPLY: input; RHS: T_old
    const double* gD;
    const double* F;
    T* y;
    const S* qs;       // [3*NQ][nc], in storage type S (converted to T on load)
    const S* cTc;      // optional per-cell
    const S* lamc;
    const S* Kq;       // per-cell K_c for a velocity formed from the head in plane()
    T cT_u, lam_u, dt, cw;
    Elem<T> e;

    // element result of the apply from the (masked) element vector u
    __device__ __forceinline__ void compute(const T (&u)[NL], long long c, T (&res)[NL]) const {
        const T cT = cTc ? cvt<T>(ldro(cTc + c)) : cT_u;
        const T dtlam = dt * (lamc ? cvt<T>(ldro(lamc + c)) : lam_u);
        core(u, u, T(1), cT, dtlam, dt * cw, c, g_nc, res);
    }
    long long g_nc;

    __device__ __forceinline__ void cell(const Grid& g, int cx, int cy, int cz, long long c,
                                         T (&res)[NL]) const {
        const T cT = cTc ? cvt<T>(ldro(cTc + c)) : cT_u;
        const T dtlam = dt * (lamc ? cvt<T>(ldro(lamc + c)) : lam_u);
        const T dtcw = dt * cw;
        const long long nc = g.nc;
        if (MODE == MODE_DIAG) {
            // mass + diffusion diagonals, then the advective diagonal
            //   sum_q W c_w N_l (q . grad N_l) = sum_d sum_q f_d(q) M^x_a M^y_b M^z_c
            // with f_d = W q_d / H_d and 1D factors B*D (direction d) or B*B,
            // contracted direction by direction (sum factorisation)
            T vol = T(1), ih[3] = {e.invH[0], e.invH[1], e.invH[2]};
            if (this->geo) {
                this->geom(c, vol, ih);
                const T i0 = ih[0] * ih[0], i1 = ih[1] * ih[1], i2 = ih[2] * ih[2];
#pragma unroll
                for (int cc = 0; cc < n; ++cc)
#pragma unroll
                    for (int b = 0; b < n; ++b)
#pragma unroll
                        for (int a = 0; a < n; ++a) {
                            const T dm = e.dm1[a] * e.dm1[b] * e.dm1[cc];
                            const T dk = e.dk1[a] * i0 * e.dm1[b] * e.dm1[cc] + e.dm1[a] * e.dk1[b] * i1 * e.dm1[cc] +
                                         e.dm1[a] * e.dm1[b] * e.dk1[cc] * i2;
                            res[a + n * (b + n * cc)] = vol * fma(dtlam, dk, cT * dm);
                        }
            } else {
#pragma unroll
                for (int l = 0; l < NL; ++l) res[l] = fma(dtlam, e.dK[l], cT * e.dM[l]);
            }
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                T f[NQ];
#pragma unroll
                for (int qi = 0; qi < NQ; ++qi)
                    f[qi] = dtcw * (e.W[qi] * vol) * ih[d] * cvt<T>(ldro(qs + (d * NQ + qi) * nc + c));
                // x: f1[qz][qy][a] = sum_qx Mx[qx][a] f[qz][qy][qx]
                T f1[NQ];
#pragma unroll
                for (int zy = 0; zy < n * n; ++zy)
#pragma unroll
                    for (int a = 0; a < n; ++a) {
                        T acc = T(0);
#pragma unroll
                        for (int qx = 0; qx < n; ++qx)
                            acc = fma(e.B[qx][a] * (d == 0 ? e.D[qx][a] : e.B[qx][a]), f[zy * n + qx], acc);
                        f1[zy * n + a] = acc;
                    }
                // y: f2[qz][b][a] = sum_qy My[qy][b] f1[qz][qy][a]
                T f2[NQ];
#pragma unroll
                for (int qz = 0; qz < n; ++qz)
#pragma unroll
                    for (int b = 0; b < n; ++b)
#pragma unroll
                        for (int a = 0; a < n; ++a) {
                            T acc = T(0);
#pragma unroll
                            for (int qy = 0; qy < n; ++qy)
                                acc = fma(e.B[qy][b] * (d == 1 ? e.D[qy][b] : e.B[qy][b]), f1[(qz * n + qy) * n + a], acc);
                            f2[(qz * n + b) * n + a] = acc;
                        }
                // z: res[c][b][a] += sum_qz Mz[qz][c] f2[qz][b][a]
#pragma unroll
                for (int c2 = 0; c2 < n; ++c2)
#pragma unroll
                    for (int ba = 0; ba < n * n; ++ba) {
                        T acc = T(0);
#pragma unroll
                        for (int qz = 0; qz < n; ++qz)
                            acc = fma(e.B[qz][c2] * (d == 2 ? e.D[qz][c2] : e.B[qz][c2]), f2[qz * n * n + ba], acc);
                        res[ba + n * n * c2] += acc;
                    }
            }
            return;
        }
        // input(s): APPLY: um = us = masked x; RHS: um = T_old - g_D, us = g_D
        if (MODE == MODE_APPLY) {
            T um[NL];
            gather<P, T>(g, x, cx, cy, cz, true, um);
            core(um, um, T(1), cT, dtlam, dtcw, c, nc, res);
        } else if (!cell_touches_dir(g, cx, cy, cz)) {
            rhs_interior(g, cx, cy, cz, res);
        } else {
            T um[NL], us[NL];
            const int i0 = P * cx, j0 = P * cy, k0 = P * cz;
#pragma unroll
            for (int c2 = 0; c2 < n; ++c2)
#pragma unroll
                for (int b = 0; b < n; ++b)
#pragma unroll
                    for (int a = 0; a < n; ++a) {
                        const int l = a + n * (b + n * c2);
                        const long long id = nidx(g, i0 + a, j0 + b, k0 + c2);
                        const bool d = on_dir(g, i0 + a, j0 + b, k0 + c2);
                        const T gv = d ? (T)gD[id] : T(0);
                        um[l] = x[id] - gv;
                        us[l] = gv;
                    }
            core(um, us, T(-1), cT, dtlam, dtcw, c, nc, res);
        }
    }

    // RHS of a cell without Dirichlet nodes: g_D vanishes on it, so only the
    // storage term cT M T_old remains; the consistent mass factors as
    // M = (G^T)^3 G^3 (the 1D mass is G^T G)
    __device__ __forceinline__ void rhs_interior(const Grid& g, int cx, int cy, int cz, T (&res)[NL]) const {
        const long long c = (long long)cx + (long long)g.ncx * ((long long)cy + (long long)g.ncy * cz);
        const T cT = cTc ? cvt<T>(ldro(cTc + c)) : cT_u;
        gather<P, T>(g, x, cx, cy, cz, false, res);
        sweep<n, 0, false>(res, e.G[0]);
        sweep<n, 1, false>(res, e.G[1]);
        sweep<n, 2, false>(res, e.G[2]);
        T sc = cT;
        if (this->geo) {
            T vol, ih[3];
            this->geom(c, vol, ih);
            sc = cT * vol;
        }
#pragma unroll
        for (int l = 0; l < NL; ++l) res[l] *= sc;
        sweep<n, 2, true>(res, e.G[2]);
        sweep<n, 1, true>(res, e.G[1]);
        sweep<n, 0, true>(res, e.G[0]);
    }

    // Contribution of Gauss plane qz to the element result of the apply
    // (cT M + dt lam K + dt C) u, written to out[l] for all (P+1)^3 l: the
    // z-sweep is restricted to plane qz and the transposed z-sweep scatters to
    // every layer; the planes' contributions add up to compute()'s result
    // (one thread per plane, u and out in shared memory).
    // With HQ the Darcy velocity q = -K_c grad h at the plane's Gauss points
    // is formed here from the head values hv of the cell (in shared memory)
    // instead of being read from qs.
    template <bool HQ = false>
    __device__ __forceinline__ void plane(const T* u, const T* hv, const long long c, const long long nc,
                                          const int qz, T* out) const {
        T vol = T(1), ih[3] = {e.invH[0], e.invH[1], e.invH[2]};
        if (this->geo) this->geom(c, vol, ih);
        const T cT = cTc ? cvt<T>(ldro(cTc + c)) : cT_u;
        const T dtlam = dt * (lamc ? cvt<T>(ldro(lamc + c)) : lam_u);
        const T dtcw = dt * cw;
        const T mK = HQ ? -cvt<T>(ldro(Kq + c)) : T(0);
        T zB[n * n], zD[n * n];
        T hzB[HQ ? n * n : 1], hzD[HQ ? n * n : 1];
#pragma unroll
        for (int ba = 0; ba < n * n; ++ba) {
            T sb = T(0), sd = T(0);
#pragma unroll
            for (int c2 = 0; c2 < n; ++c2) {
                const T uv = u[ba + n * n * c2];
                sb = fma(e.B[qz][c2], uv, sb);
                sd = fma(e.D[qz][c2], uv, sd);
            }
            zB[ba] = sb;
            zD[ba] = sd;
            if (HQ) {
                T hb = T(0), hd = T(0);
#pragma unroll
                for (int c2 = 0; c2 < n; ++c2) {
                    const T hh = hv[ba + n * n * c2];
                    hb = fma(e.B[qz][c2], hh, hb);
                    hd = fma(e.D[qz][c2], hh, hd);
                }
                hzB[ba] = hb;
                hzD[ba] = hd;
            }
        }
        T s1[n * n], s2[n * n];
#pragma unroll
        for (int ba = 0; ba < n * n; ++ba) { s1[ba] = T(0); s2[ba] = T(0); }
#pragma unroll 1   // rolled: fewer live registers per plane thread (measured faster)
        for (int qy = 0; qy < n; ++qy) {
            T yBB[n], yDB[n], yBD[n];
            T hBB[HQ ? n : 1], hDB[HQ ? n : 1], hBD[HQ ? n : 1];
#pragma unroll
            for (int a = 0; a < n; ++a) {
                T v0 = T(0), v2 = T(0), v3 = T(0);
#pragma unroll
                for (int b = 0; b < n; ++b) {
                    v0 = fma(e.B[qy][b], zB[a + n * b], v0);
                    v2 = fma(e.D[qy][b], zB[a + n * b], v2);
                    v3 = fma(e.B[qy][b], zD[a + n * b], v3);
                }
                yBB[a] = v0; yDB[a] = v2; yBD[a] = v3;
                if (HQ) {
                    T w0 = T(0), w2 = T(0), w3 = T(0);
#pragma unroll
                    for (int b = 0; b < n; ++b) {
                        w0 = fma(e.B[qy][b], hzB[a + n * b], w0);
                        w2 = fma(e.D[qy][b], hzB[a + n * b], w2);
                        w3 = fma(e.B[qy][b], hzD[a + n * b], w3);
                    }
                    hBB[a] = w0; hDB[a] = w2; hBD[a] = w3;
                }
            }
            T t1[n], t2[n], t3[n];
#pragma unroll
            for (int a = 0; a < n; ++a) { t1[a] = T(0); t2[a] = T(0); t3[a] = T(0); }
#pragma unroll
            for (int qx = 0; qx < n; ++qx) {
                T val = T(0), gx = T(0), gy = T(0), gz = T(0);
#pragma unroll
                for (int a = 0; a < n; ++a) {
                    val = fma(e.B[qx][a], yBB[a], val);
                    gx = fma(e.D[qx][a], yBB[a], gx);
                    gy = fma(e.B[qx][a], yDB[a], gy);
                    gz = fma(e.B[qx][a], yBD[a], gz);
                }
                gx *= ih[0];
                gy *= ih[1];
                gz *= ih[2];
                const int qi = qx + n * (qy + n * qz);
                T q0, q1, q2;
                if (HQ) {
                    T hx = T(0), hy = T(0), hz = T(0);
#pragma unroll
                    for (int a = 0; a < n; ++a) {
                        hx = fma(e.D[qx][a], hBB[a], hx);
                        hy = fma(e.B[qx][a], hDB[a], hy);
                        hz = fma(e.B[qx][a], hBD[a], hz);
                    }
                    q0 = mK * (hx * ih[0]);
                    q1 = mK * (hy * ih[1]);
                    q2 = mK * (hz * ih[2]);
                } else {
                    q0 = cvt<T>(ldro(qs + (0 * NQ + qi) * nc + c));
                    q1 = cvt<T>(ldro(qs + (1 * NQ + qi) * nc + c));
                    q2 = cvt<T>(ldro(qs + (2 * NQ + qi) * nc + c));
                }
                const T W = (e.W[qi] * vol);
                const T v = W * fma(cT, val, dtcw * (q0 * gx + q1 * gy + q2 * gz));
                const T f = W * dtlam;
                const T gxs = f * gx * ih[0];
                const T gys = f * gy * ih[1];
                const T gzs = f * gz * ih[2];
#pragma unroll
                for (int a = 0; a < n; ++a) {
                    t1[a] = fma(e.B[qx][a], v, fma(e.D[qx][a], gxs, t1[a]));
                    t2[a] = fma(e.B[qx][a], gys, t2[a]);
                    t3[a] = fma(e.B[qx][a], gzs, t3[a]);
                }
            }
#pragma unroll
            for (int b = 0; b < n; ++b)
#pragma unroll
                for (int a = 0; a < n; ++a) {
                    s1[a + n * b] = fma(e.B[qy][b], t1[a], fma(e.D[qy][b], t2[a], s1[a + n * b]));
                    s2[a + n * b] = fma(e.B[qy][b], t3[a], s2[a + n * b]);
                }
        }
#pragma unroll
        for (int c2 = 0; c2 < n; ++c2)
#pragma unroll
            for (int ba = 0; ba < n * n; ++ba)
                out[ba + n * n * c2] = fma(e.B[qz][c2], s1[ba], e.D[qz][c2] * s2[ba]);
    }

    // sum-factorised quadrature: res = cT M um + sgn (dt lam K + dt C) us
    __device__ __forceinline__ void core(const T (&um)[NL], const T (&us)[NL], const T sgn,
                                         const T cT, const T dtlam, const T dtcw, const long long c,
                                         const long long nc, T (&res)[NL]) const {
        T vol = T(1), ih[3] = {e.invH[0], e.invH[1], e.invH[2]};
        if (this->geo) this->geom(c, vol, ih);
#pragma unroll
        for (int l = 0; l < NL; ++l) res[l] = T(0);
#pragma unroll
        for (int qz = 0; qz < n; ++qz) {
            // z sweep
            T zBm[n * n], zBs[n * n], zDs[n * n];
#pragma unroll
            for (int ba = 0; ba < n * n; ++ba) {
                T sm = T(0), sb = T(0), sd = T(0);
#pragma unroll
                for (int c2 = 0; c2 < n; ++c2) {
                    sm = fma(e.B[qz][c2], um[ba + n * n * c2], sm);
                    sb = fma(e.B[qz][c2], us[ba + n * n * c2], sb);
                    sd = fma(e.D[qz][c2], us[ba + n * n * c2], sd);
                }
                zBm[ba] = sm;
                zBs[ba] = sb;
                zDs[ba] = sd;
            }
            T s1[n * n], s2[n * n];
#pragma unroll
            for (int ba = 0; ba < n * n; ++ba) { s1[ba] = T(0); s2[ba] = T(0); }
#pragma unroll
            for (int qy = 0; qy < n; ++qy) {
                T yBBm[n], yBBs[n], yDBs[n], yBDs[n];
#pragma unroll
                for (int a = 0; a < n; ++a) {
                    T v0 = T(0), v1 = T(0), v2 = T(0), v3 = T(0);
#pragma unroll
                    for (int b = 0; b < n; ++b) {
                        v0 = fma(e.B[qy][b], zBm[a + n * b], v0);
                        v1 = fma(e.B[qy][b], zBs[a + n * b], v1);
                        v2 = fma(e.D[qy][b], zBs[a + n * b], v2);
                        v3 = fma(e.B[qy][b], zDs[a + n * b], v3);
                    }
                    yBBm[a] = v0; yBBs[a] = v1; yDBs[a] = v2; yBDs[a] = v3;
                }
                T t1[n], t2[n], t3[n];
#pragma unroll
                for (int a = 0; a < n; ++a) { t1[a] = T(0); t2[a] = T(0); t3[a] = T(0); }
#pragma unroll
                for (int qx = 0; qx < n; ++qx) {
                    T val = T(0), gx = T(0), gy = T(0), gz = T(0);
#pragma unroll
                    for (int a = 0; a < n; ++a) {
                        val = fma(e.B[qx][a], yBBm[a], val);
                        gx = fma(e.D[qx][a], yBBs[a], gx);
                        gy = fma(e.B[qx][a], yDBs[a], gy);
                        gz = fma(e.B[qx][a], yBDs[a], gz);
                    }
                    gx *= ih[0];
                    gy *= ih[1];
                    gz *= ih[2];
                    const int qi = qx + n * (qy + n * qz);
                    const T q0 = cvt<T>(ldro(qs + (0 * NQ + qi) * nc + c));
                    const T q1 = cvt<T>(ldro(qs + (1 * NQ + qi) * nc + c));
                    const T q2 = cvt<T>(ldro(qs + (2 * NQ + qi) * nc + c));
                    const T W = (e.W[qi] * vol);
                    const T v = W * fma(cT, val, sgn * dtcw * (q0 * gx + q1 * gy + q2 * gz));
                    const T f = sgn * W * dtlam;
                    const T gxs = f * gx * ih[0];
                    const T gys = f * gy * ih[1];
                    const T gzs = f * gz * ih[2];
#pragma unroll
                    for (int a = 0; a < n; ++a) {
                        t1[a] = fma(e.B[qx][a], v, fma(e.D[qx][a], gxs, t1[a]));
                        t2[a] = fma(e.B[qx][a], gys, t2[a]);
                        t3[a] = fma(e.B[qx][a], gzs, t3[a]);
                    }
                }
#pragma unroll
                for (int b = 0; b < n; ++b)
#pragma unroll
                    for (int a = 0; a < n; ++a) {
                        s1[a + n * b] = fma(e.B[qy][b], t1[a], fma(e.D[qy][b], t2[a], s1[a + n * b]));
                        s2[a + n * b] = fma(e.B[qy][b], t3[a], s2[a + n * b]);
                    }
            }
#pragma unroll
            for (int c2 = 0; c2 < n; ++c2)
#pragma unroll
                for (int ba = 0; ba < n * n; ++ba)
                    res[ba + n * n * c2] =
                        fma(e.B[qz][c2], s1[ba], fma(e.D[qz][c2], s2[ba], res[ba + n * n * c2]));
        }
    }

    __device__ __forceinline__ void emit(const Grid& g, int i, int j, int k, T val, T& dot) const {
        const long long id = nidx(g, i, j, k);
        const bool d = on_dir(g, i, j, k);
        if (MODE == MODE_APPLY) {
            const T xv = x[id];
            const T yv = d ? xv : val;
            y[id] = yv;
            dot = fma(xv, yv, dot);
        } else if (MODE == MODE_RHS) {
            y[id] = d ? (T)gD[id] : val + dt * (T)F[id];
        } else {
            y[id] = d ? T(1) : val;
        }
    }
};

// ---------------------------------------------------------------------------
// The tile kernel
// ---------------------------------------------------------------------------
template <int P, int CXM, int CYM>
struct TileShape {
    static constexpr int TX = P * (CXM - 1), TY = P * (CYM - 1), NT = CXM * CYM;
    static constexpr int CPT = (TX * TY + NT - 1) / NT;
};

template <int P, typename T, int CXM, int CYM, class Op>
__global__ void __launch_bounds__(CXM* CYM) tile_kernel(const Grid g, const Op op, const int ZC,
                                                        double* __restrict__ dot_part,
                                                        const Scal* __restrict__ sc) {
    if (sc && sc->done) return;
    using S = TileShape<P, CXM, CYM>;
    constexpr int n = P + 1, NL = n * n * n;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* E = reinterpret_cast<T*>(smem_raw);

    const int ix0 = blockIdx.x * S::TX, iy0 = blockIdx.y * S::TY;
    const int ix1 = min(ix0 + S::TX, g.Nx), iy1 = min(iy0 + S::TY, g.Ny);
    const int cx_lo = max(ix0 / P - 1, 0), cy_lo = max(iy0 / P - 1, 0);
    const int cx_hi = min((ix1 - 1) / P, g.ncx - 1), cy_hi = min((iy1 - 1) / P, g.ncy - 1);
    const int CX = cx_hi - cx_lo + 1, CY = cy_hi - cy_lo + 1;
    const int TXo = ix1 - ix0, TYo = iy1 - iy0;
    const int last = (blockIdx.z == gridDim.z - 1);
    const int k0 = blockIdx.z * ZC * P;
    const int k1 = last ? g.Nz : min(k0 + ZC * P, g.Nz);
    const int cz_lo = max((int)blockIdx.z * ZC - 1, 0);
    const int cz_hi = last ? g.ncz - 1 : min((int)blockIdx.z * ZC + ZC - 1, g.ncz - 1);

    T carry[S::CPT];
#pragma unroll
    for (int s = 0; s < S::CPT; ++s) carry[s] = T(0);
    T dot = T(0);

    for (int cz = cz_lo; cz <= cz_hi; ++cz) {
        {
            const int cidx = threadIdx.x;
            if (cidx < CX * CY) {
                const int lx = cidx % CX, ly = cidx / CX;
                const int cx = cx_lo + lx, cy = cy_lo + ly;
                const long long c = (long long)cx + (long long)g.ncx * ((long long)cy + (long long)g.ncy * cz);
                T res[NL];
                op.cell(g, cx, cy, cz, c, res);
                T* e = E + (size_t)cidx * NL;
#pragma unroll
                for (int l = 0; l < NL; ++l) e[l] = res[l];
            }
        }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < S::CPT; ++s) {
            const int col = threadIdx.x + s * S::NT;
            if (col < TXo * TYo) {
                const int ix = ix0 + col % TXo, iy = iy0 + col / TXo;
                int cxs[2], axs[2], ncxs = 0, cys[2], bys[2], ncys = 0;
                if (ix % P == 0) {
                    if (ix / P - 1 >= 0) { cxs[ncxs] = ix / P - 1; axs[ncxs++] = P; }
                    if (ix / P < g.ncx) { cxs[ncxs] = ix / P; axs[ncxs++] = 0; }
                } else { cxs[0] = ix / P; axs[0] = ix % P; ncxs = 1; }
                if (iy % P == 0) {
                    if (iy / P - 1 >= 0) { cys[ncys] = iy / P - 1; bys[ncys++] = P; }
                    if (iy / P < g.ncy) { cys[ncys] = iy / P; bys[ncys++] = 0; }
                } else { cys[0] = iy / P; bys[0] = iy % P; ncys = 1; }
                T sj[P + 1];
#pragma unroll
                for (int j = 0; j <= P; ++j) sj[j] = T(0);
                for (int yy = 0; yy < ncys; ++yy)
                    for (int xx = 0; xx < ncxs; ++xx) {
                        const T* base = E + (size_t)((cxs[xx] - cx_lo) + CX * (cys[yy] - cy_lo)) * NL +
                                        axs[xx] + n * bys[yy];
#pragma unroll
                        for (int j = 0; j <= P; ++j) sj[j] += base[n * n * j];
                    }
                const int kb = P * cz;
                if (kb >= k0 && kb < k1) op.emit(g, ix, iy, kb, carry[s] + sj[0], dot);
#pragma unroll
                for (int j = 1; j < P; ++j)
                    if (kb + j >= k0 && kb + j < k1) op.emit(g, ix, iy, kb + j, sj[j], dot);
                carry[s] = sj[P];
                if (cz == g.ncz - 1 && kb + P >= k0 && kb + P < k1) op.emit(g, ix, iy, kb + P, carry[s], dot);
            }
        }
        __syncthreads();
    }
    if (dot_part) {
        const double tot = block_sum_t(dot);
        if (threadIdx.x == 0)
            dot_part[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = tot;
    }
}


// ---------------------------------------------------------------------------
// The operator-apply kernel: like tile_kernel, but the node planes of each
// cell layer are staged in shared memory by asynchronous copies (cp.async,
// zero-filled for Dirichlet nodes) issued one layer ahead of the compute, so
// every node value is read from global memory once per tile and the copies
// of layer cz+1 overlap the cell work of layer cz.
//   shared memory: slab [2P+1 plane slots][P*CYM+1][P*CXM+1] of T, then the
//   element results E [CXM*CYM][(P+1)^3].
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async_elem(void* dst, const void* src, int bytes, int src_bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if (bytes == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes));
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::); }

template <int P, int CXM, int CYM, typename T>
struct ApplySmem {
    static constexpr int n = P + 1, NL = n * n * n;
    static constexpr int SX = P * CXM + 1, SY = P * CYM + 1, NS = 2 * P + 1;
    static constexpr size_t slab_elems = (size_t)NS * SX * SY;
    static constexpr size_t bytes = (slab_elems + (size_t)CXM * CYM * NL) * sizeof(T);
};

template <int P, typename T, int CXM, int CYM, class Op>
__global__ void __launch_bounds__(CXM* CYM) apply_kernel(const Grid g, const Op op, const int ZC,
                                                         const T* __restrict__ x, T* __restrict__ y,
                                                         double* __restrict__ dot_part,
                                                         const Scal* __restrict__ sc) {
    if (sc && sc->done) return;
    using S = TileShape<P, CXM, CYM>;
    using M = ApplySmem<P, CXM, CYM, T>;
    constexpr int n = P + 1, NL = n * n * n;
    constexpr int SX = M::SX, SY = M::SY, NS = M::NS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* slab = reinterpret_cast<T*>(smem_raw);
    T* E = slab + M::slab_elems;

    const int ix0 = blockIdx.x * S::TX, iy0 = blockIdx.y * S::TY;
    const int ix1 = min(ix0 + S::TX, g.Nx), iy1 = min(iy0 + S::TY, g.Ny);
    const int cx_lo = max(ix0 / P - 1, 0), cy_lo = max(iy0 / P - 1, 0);
    const int cx_hi = min((ix1 - 1) / P, g.ncx - 1), cy_hi = min((iy1 - 1) / P, g.ncy - 1);
    const int CX = cx_hi - cx_lo + 1, CY = cy_hi - cy_lo + 1;
    const int TXo = ix1 - ix0, TYo = iy1 - iy0;
    const int last = (blockIdx.z == gridDim.z - 1);
    const int k0 = blockIdx.z * ZC * P;
    const int k1 = last ? g.Nz : min(k0 + ZC * P, g.Nz);
    const int cz_lo = max((int)blockIdx.z * ZC - 1, 0);
    const int cz_hi = last ? g.ncz - 1 : min((int)blockIdx.z * ZC + ZC - 1, g.ncz - 1);
    const int i0 = P * cx_lo, j0 = P * cy_lo;
    const int NXs = P * CX + 1, NYs = P * CY + 1;
    const int plane = g.Nx * g.Ny;           // node counts fit in 32 bits
    const bool tile_dir = g.dmask != 0 &&
                          ((cx_lo == 0 && (g.dmask & 1)) || (cx_hi == g.ncx - 1 && (g.dmask & 2)) ||
                           (cy_lo == 0 && (g.dmask & 4)) || (cy_hi == g.ncy - 1 && (g.dmask & 8)) ||
                           (cz_lo == 0 && (g.dmask & 16)) || (cz_hi == g.ncz - 1 && (g.dmask & 32)));

    // copies of node planes ka..kb into their slots (k mod NS), one row per
    // warp and one node per lane; Dirichlet nodes are zero-filled
    auto issue = [&](int ka, int kb) {
        const int rows = (kb - ka + 1) * NYs;
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int r = wid; r < rows; r += nw) {
            const int pl = r / NYs, ly = r - pl * NYs;
            const int k = ka + pl, j = j0 + ly;
            T* drow = slab + ((k % NS) * SY + ly) * SX;
            const T* srow = x + (g.Nx * j + plane * k);
            const bool rowdir = tile_dir && (((g.dmask & 4) && j == 0) || ((g.dmask & 8) && j == g.Ny - 1) ||
                                             ((g.dmask & 16) && k == 0) || ((g.dmask & 32) && k == g.Nz - 1));
            for (int lx = lane; lx < NXs; lx += 32) {
                const int i = i0 + lx;
                const bool z = rowdir || (tile_dir && (((g.dmask & 1) && i == 0) || ((g.dmask & 2) && i == g.Nx - 1)));
                cp_async_elem(drow + lx, srow + i, (int)sizeof(T), z ? 0 : (int)sizeof(T));
            }
        }
        cp_async_commit();
    };

    // per owned column: element-result offsets of its (up to 4) cells, slot
    // xx + 2*yy for the lower/upper neighbour cell in x / y (-1: none)
    int offs[S::CPT][4], gcol[S::CPT];
#pragma unroll
    for (int s = 0; s < S::CPT; ++s) {
        gcol[s] = -1;
#pragma unroll
        for (int q = 0; q < 4; ++q) offs[s][q] = -1;
        const int col = threadIdx.x + s * S::NT;
        if (col < TXo * TYo) {
            const int ix = ix0 + col % TXo, iy = iy0 + col / TXo;
            int cxs[2] = {-1, -1}, axs[2] = {0, 0}, cys[2] = {-1, -1}, bys[2] = {0, 0};
            if (ix % P == 0) {
                if (ix / P - 1 >= 0) { cxs[0] = ix / P - 1; axs[0] = P; }
                if (ix / P < g.ncx) { cxs[1] = ix / P; axs[1] = 0; }
            } else { cxs[0] = ix / P; axs[0] = ix % P; }
            if (iy % P == 0) {
                if (iy / P - 1 >= 0) { cys[0] = iy / P - 1; bys[0] = P; }
                if (iy / P < g.ncy) { cys[1] = iy / P; bys[1] = 0; }
            } else { cys[0] = iy / P; bys[0] = iy % P; }
#pragma unroll
            for (int yy = 0; yy < 2; ++yy)
#pragma unroll
                for (int xx = 0; xx < 2; ++xx)
                    if (cxs[xx] >= 0 && cys[yy] >= 0)
                        offs[s][xx + 2 * yy] = ((cxs[xx] - cx_lo) + CX * (cys[yy] - cy_lo)) * NL + axs[xx] + n * bys[yy];
            gcol[s] = ix + g.Nx * iy;
        }
    }

    T carry[S::CPT];
#pragma unroll
    for (int s = 0; s < S::CPT; ++s) carry[s] = T(0);
    T dot = T(0);

    issue(P * cz_lo, P * cz_lo + P);
    for (int cz = cz_lo; cz <= cz_hi; ++cz) {
        if (cz < cz_hi) issue(P * cz + P + 1, P * cz + 2 * P);
        else cp_async_commit();
        cp_async_wait_1();
        __syncthreads();
        {
            const int cidx = threadIdx.x;
            if (cidx < CX * CY) {
                const int lx = cidx % CX, ly = cidx / CX;
                const long long c = (long long)(cx_lo + lx) + (long long)g.ncx * ((cy_lo + ly) + (long long)g.ncy * cz);
                T u[NL];
#pragma unroll
                for (int c2 = 0; c2 < n; ++c2) {
                    const T* pl = slab + ((P * cz + c2) % NS) * SY * SX;
#pragma unroll
                    for (int b = 0; b < n; ++b)
#pragma unroll
                        for (int a = 0; a < n; ++a) u[a + n * (b + n * c2)] = pl[(P * ly + b) * SX + P * lx + a];
                }
                T res[NL];
                op.compute(u, c, res);
                T* e = E + (size_t)cidx * NL;
#pragma unroll
                for (int l = 0; l < NL; ++l) e[l] = res[l];
            }
        }
        __syncthreads();
        const int kb = P * cz;
#pragma unroll
        for (int s = 0; s < S::CPT; ++s) {
            if (gcol[s] < 0) continue;
            T sj[P + 1];
#pragma unroll
            for (int j = 0; j <= P; ++j) sj[j] = T(0);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (offs[s][q] < 0) continue;
                const T* base = E + offs[s][q];
#pragma unroll
                for (int j = 0; j <= P; ++j) sj[j] += base[n * n * j];
            }
            const int col = threadIdx.x + s * S::NT;
            const int lxn = ix0 + col % TXo - i0, lyn = iy0 + col / TXo - j0;
#pragma unroll
            for (int j = 0; j <= P; ++j) {
                const int k = kb + j;
                T val;
                bool emit_it;
                if (j == 0) { val = carry[s] + sj[0]; emit_it = k >= k0 && k < k1; }
                else if (j < P) { val = sj[j]; emit_it = k >= k0 && k < k1; }
                else { carry[s] = sj[P]; val = carry[s]; emit_it = (cz == g.ncz - 1) && k >= k0 && k < k1; }
                if (emit_it) {
                    const int id = gcol[s] + plane * k;
                    T xv = slab[((k % NS) * SY + lyn) * SX + lxn];
                    T yv = val;
                    if (tile_dir && on_dir(g, ix0 + col % TXo, iy0 + col / TXo, k)) {
                        xv = x[id];   // Dirichlet row: identity, unmasked value
                        yv = xv;
                    }
                    y[id] = yv;
                    dot = fma(xv, yv, dot);
                }
            }
        }
        __syncthreads();
    }
    if (dot_part) {
        const double tot = block_sum_t(dot);
        if (threadIdx.x == 0)
            dot_part[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = tot;
    }
}


// ---------------------------------------------------------------------------
// Two-pass operator apply (variant used for FP32): pass 1 computes every
// cell once (one thread per cell, no barriers) into an element-result buffer
// E laid out component-major, E[l * nc + c], which stays in L2 for the mesh
// sizes of interest; pass 2 gives every node its own thread, which sums the
// contributions of its cells in a fixed order (deterministic, no atomics),
// applies the Dirichlet identity rows and accumulates the fused dot product.
// ---------------------------------------------------------------------------
// Thread (cx, cy) of a (32 x 4) block marches through its share of the cell
// layers; all indices are 32-bit and advance incrementally.
template <int P, typename T, class Op>
__global__ void __launch_bounds__(128) cell_pass_kernel(const Grid g, const Op op, const T* __restrict__ x,
                                                        T* __restrict__ E, const int zlen,
                                                        const Scal* __restrict__ sc) {
    if (sc && sc->done) return;
    constexpr int n = P + 1, NL = n * n * n;
    const int cx = blockIdx.x * blockDim.x + threadIdx.x;
    const int cy = blockIdx.y * blockDim.y + threadIdx.y;
    if (cx >= g.ncx || cy >= g.ncy) return;
    const int cz0 = blockIdx.z * zlen, cz1 = min(cz0 + zlen, g.ncz);
    const int nc = (int)g.nc, layer = g.ncx * g.ncy;
    const int NX = g.Nx, NXY = g.Nx * g.Ny;
    int off[n * n];   // offsets of the (b, c) node rows of a cell
#pragma unroll
    for (int c2 = 0; c2 < n; ++c2)
#pragma unroll
        for (int b = 0; b < n; ++b) off[b + n * c2] = NX * b + NXY * c2;
    const bool edge_xy = g.dmask != 0 && (cx == 0 || cx == g.ncx - 1 || cy == 0 || cy == g.ncy - 1);
    int base = P * cx + NX * P * cy + NXY * P * cz0;
    int c = cx + g.ncx * cy + layer * cz0;
    for (int cz = cz0; cz < cz1; ++cz, base += NXY * P, c += layer) {
        T u[NL];
#pragma unroll
        for (int bc = 0; bc < n * n; ++bc)
#pragma unroll
            for (int a2 = 0; a2 < n; ++a2) u[a2 + n * bc] = ldro(x + base + off[bc] + a2);
        if (edge_xy || (g.dmask & 48 && (cz == 0 || cz == g.ncz - 1))) {
#pragma unroll
            for (int c2 = 0; c2 < n; ++c2)
#pragma unroll
                for (int b = 0; b < n; ++b)
#pragma unroll
                    for (int a2 = 0; a2 < n; ++a2)
                        if (on_dir(g, P * cx + a2, P * cy + b, P * cz + c2)) u[a2 + n * (b + n * c2)] = T(0);
        }
        T res[NL];
        op.compute(u, c, res);
#pragma unroll
        for (int l = 0; l < NL; ++l) E[l * nc + c] = res[l];
    }
}

// The element contributions of node (i, j, k): up to 2 x 2 x 2 cells share
// it.  E[l * nc + c] splits into an xy part fixed per thread (eb[q] for the 4
// cell columns q = xx + 2 yy around the node) and a z part that is the same
// for every node of a layer (ez[zz] for the cell layers below and above).
template <int P>
struct NodeXY {
    int eb[4];
    bool vxy[4];
    bool dir;
    __device__ __forceinline__ NodeXY(const Grid& g, int i, int j) {
        constexpr int n = P + 1;
        const int nc = (int)g.nc;
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
                eb[q] = (axs[xx] + n * bys[yy]) * nc + cxs[xx] + g.ncx * cys[yy];
            }
        dir = ((g.dmask & 1) && i == 0) || ((g.dmask & 2) && i == g.Nx - 1) ||
              ((g.dmask & 4) && j == 0) || ((g.dmask & 8) && j == g.Ny - 1);
    }

    // the 8 element contributions at node layer k; an absent one (no cell on
    // that side) reads the zero slot E[-1] in front of the element buffer, so
    // every load is unconditional
    template <typename T>
    __device__ __forceinline__ void load(const Grid& g, const T* __restrict__ E, int k, T (&v)[8]) const {
        constexpr int n = P + 1;
        const int nc = (int)g.nc, layer = g.ncx * g.ncy;
        int ez[2];
        bool vz[2];
        if (k % P == 0) {
            ez[0] = n * n * P * nc + layer * (k / P - 1);
            vz[0] = k > 0;
            ez[1] = layer * (k / P);
            vz[1] = k / P < g.ncz;
        } else {
            ez[0] = n * n * (k % P) * nc + layer * (k / P);
            vz[0] = true;
            ez[1] = 0;
            vz[1] = false;
        }
#pragma unroll
        for (int zz = 0; zz < 2; ++zz)
#pragma unroll
            for (int q = 0; q < 4; ++q)
                v[q + 4 * zz] = ldg_any(E + ((vz[zz] && vxy[q]) ? eb[q] + ez[zz] : -1));
    }
};

// Node pass of the two-pass apply: y = sum of the element contributions at
// each node in a fixed order (x at Dirichlet nodes), optional partial sums of
// x.y.  128 nodes of a layer per CTA (a linear run of node indices, so the
// vector accesses are coalesced), each thread marching klen layers two at a
// time so that twice the loads are in flight.
template <int P, typename T>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 12 : 1) node_pass_kernel(const Grid g, const T* __restrict__ E,
                                                        const T* __restrict__ x, T* __restrict__ y,
                                                        const int klen, double* __restrict__ dot_part,
                                                        const Scal* __restrict__ sc) {
    if (sc && sc->done) return;
    const int NXY = g.Nx * g.Ny;
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    T dot = T(0);
    if (m < NXY) {
        const NodeXY<P> nx(g, m % g.Nx, m / g.Nx);
        const int k0 = blockIdx.y * klen, k1 = min(k0 + klen, g.Nz);
        auto finish = [&](int k, int id, const T (&v)[8], T xv) {
            const bool d = nx.dir || ((g.dmask & 16) && k == 0) || ((g.dmask & 32) && k == g.Nz - 1);
            const T sum = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
            const T yv = d ? xv : sum;
            y[id] = yv;
            dot = fma(xv, yv, dot);
        };
        int k = k0, id = m + NXY * k0;
        for (; k + 1 < k1; k += 2, id += 2 * NXY) {
            T v0[8], v1[8];
            nx.load(g, E, k, v0);
            nx.load(g, E, k + 1, v1);
            const T x0 = x[id], x1 = x[id + NXY];
            finish(k, id, v0, x0);
            finish(k + 1, id + NXY, v1, x1);
        }
        if (k < k1) {
            T v0[8];
            nx.load(g, E, k, v0);
            finish(k, id, v0, x[id]);
        }
    }
    if (dot_part) {
        const double tot = block_sum_t(dot);
        if (threadIdx.x == 0) dot_part[blockIdx.x + gridDim.x * blockIdx.y] = tot;
    }
}

// ---------------------------------------------------------------------------
// Fused Jacobi-CG iteration over the two-pass apply (head operator), two
// launches per iteration:
//   cell pass:  p_e = Dinv r + beta p_old at the cell's nodes (Dirichlet
//               nodes zero), E = A_e p_e, partial of sum_e p_e . A_e p_e;
//               the last CTA to finish reduces the partials in a fixed order
//               and sets alpha = r.z / p.Ap (or flags a breakdown).
//   node pass:  q = sum of the element contributions, p = Dinv r + beta p_old
//               (the same formula, so the same value), x += alpha p,
//               r -= alpha q; partials of r.Dinv.r and r.r; the last CTA
//               reduces them, tests convergence and sets beta for the next
//               iteration.
// A CTA learns that it is last from an atomic ticket in s (the classic
// threadfence reduction): no CTA waits for another, and the sums do not
// depend on the order in which CTAs finish.
// ---------------------------------------------------------------------------

// Column march of the fused Krylov cell passes: thread (cx, cy) walks cells
// cz0..cz1 of its column, forms the operator input at the cell's nodes with
// nv(id) (Dirichlet nodes zero), writes E = A_e u and returns sum_e u . A_e u
// when DOT.  The bottom face of a cell is the top face of the cell below (the
// same nodes, so the same values): it is carried, not re-read.
template <int P, typename T, class Op, class NV, bool DOT>
__device__ __forceinline__ T march_cells(const Grid& g, const Op& op, const NV& nv, T* __restrict__ E,
                                         const int zlen) {
    constexpr int n = P + 1, NL = n * n * n, NF = n * n;
    const int cx = blockIdx.x * blockDim.x + threadIdx.x;
    const int cy = blockIdx.y * blockDim.y + threadIdx.y;
    T dot = T(0);
    if (cx >= g.ncx || cy >= g.ncy) return dot;
    const int cz0 = blockIdx.z * zlen, cz1 = min(cz0 + zlen, g.ncz);
    const int nc = (int)g.nc, layer = g.ncx * g.ncy;
    const int NX = g.Nx, NXY = g.Nx * g.Ny;
    const bool edge_xy = g.dmask != 0 && (cx == 0 || cx == g.ncx - 1 || cy == 0 || cy == g.ncy - 1);
    int base = P * cx + NX * P * cy + NXY * P * cz0;
    int c = cx + g.ncx * cy + layer * cz0;
    T carry[NF];
#pragma unroll
    for (int b = 0; b < n; ++b)
#pragma unroll
        for (int a = 0; a < n; ++a) carry[a + n * b] = nv(base + NX * b + a);
    for (int cz = cz0; cz < cz1; ++cz, base += NXY * P, c += layer) {
        T u[NL];
#pragma unroll
        for (int f = 0; f < NF; ++f) u[f] = carry[f];
#pragma unroll
        for (int c2 = 1; c2 < n; ++c2)
#pragma unroll
            for (int b = 0; b < n; ++b)
#pragma unroll
                for (int a = 0; a < n; ++a) u[a + n * (b + n * c2)] = nv(base + NX * b + NXY * c2 + a);
        if (edge_xy || (g.dmask & 48 && (cz == 0 || cz == g.ncz - 1))) {
#pragma unroll
            for (int c2 = 0; c2 < n; ++c2)
#pragma unroll
                for (int b = 0; b < n; ++b)
#pragma unroll
                    for (int a = 0; a < n; ++a)
                        if (on_dir(g, P * cx + a, P * cy + b, P * cz + c2)) u[a + n * (b + n * c2)] = T(0);
        }
        // the top face becomes the next bottom face; a node zeroed as a
        // Dirichlet node is zero in the next cell too
#pragma unroll
        for (int f = 0; f < NF; ++f) carry[f] = u[f + NF * P];
        if (DOT) {
            op.compute_dot_inplace(u, c, dot);
        } else {
            T res[NL];
            op.compute(u, c, res);
#pragma unroll
            for (int l = 0; l < NL; ++l) u[l] = res[l];
        }
#pragma unroll
        for (int l = 0; l < NL; ++l) E[l * nc + c] = u[l];
    }
    return dot;
}

// CG search direction at a node: p = Dinv r + beta p_old
template <typename T>
struct CgDir {
    const T* r;
    const T* Dinv;
    const T* p;
    T beta;
    __device__ __forceinline__ T operator()(int id) const { return fma(beta, ldro(p + id), ldro(Dinv + id) * ldro(r + id)); }
};

template <int P, typename T, class Op>
__global__ void __launch_bounds__(128) fcg_cell_kernel(const Grid g, const Op op, const T* __restrict__ r,
                                                       const T* __restrict__ Dinv, const T* __restrict__ p,
                                                       T* __restrict__ E, const int zlen, Scal* s,
                                                       double* __restrict__ part, const int first) {
    if (s->done) return;
    const CgDir<T> nv{r, Dinv, p, first ? T(0) : (T)s->beta};
    const T pap = march_cells<P, T, Op, CgDir<T>, true>(g, op, nv, E, zlen);
    const double v = block_sum_t(pap);
    const unsigned nblk = gridDim.x * gridDim.y * gridDim.z;
    if (!publish_and_ticket(s, part, &v, 1, 0, nblk)) return;
    const double tot = last_cta_sum(part, (int)nblk);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        s->ticket = 0;
        s->pq = tot;
        if (!(tot > 0.0) || !isfinite(tot)) { s->status = ST_BREAKDOWN; s->done = 1; }
        else s->alpha = s->rz / tot;
    }
}

// node pass of the fused CG: 128 nodes of a layer per CTA (a linear run of
// node indices, so the vector accesses are fully coalesced), each thread
// marching klen layers two at a time so that twice the loads are in flight
template <int P, typename T>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 12 : 1) fcg_node_kernel(const Grid g, const T* __restrict__ E, T* __restrict__ x,
                                                       T* __restrict__ r, const T* __restrict__ Dinv,
                                                       T* __restrict__ p, const int klen, Scal* s,
                                                       double* __restrict__ part, const int stride,
                                                       const int first) {
    if (s->done) return;
    const T alpha = (T)s->alpha;
    const T beta = first ? T(0) : (T)s->beta;
    const int NXY = g.Nx * g.Ny;
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    T rzp = T(0), rrp = T(0);
    if (m < NXY) {
        const NodeXY<P> nx(g, m % g.Nx, m / g.Nx);
        const int k0 = blockIdx.y * klen, k1 = min(k0 + klen, g.Nz);
        auto finish = [&](int k, int id, const T (&v)[8], T di, T ri, T pi, T xi) {
            const bool d = nx.dir || ((g.dmask & 16) && k == 0) || ((g.dmask & 32) && k == g.Nz - 1);
            T pn = fma(beta, pi, di * ri);
            if (d) pn = T(0);
            const T q = d ? pn : ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
            p[id] = pn;
            x[id] = fma(alpha, pn, xi);
            const T rn = fma(-alpha, q, ri);
            r[id] = rn;
            rzp = fma(rn, di * rn, rzp);
            rrp = fma(rn, rn, rrp);
        };
        int k = k0, id = m + NXY * k0;
        for (; k + 1 < k1; k += 2, id += 2 * NXY) {
            T v0[8], v1[8];
            nx.load(g, E, k, v0);
            nx.load(g, E, k + 1, v1);
            const T d0 = Dinv[id], r0 = r[id], p0 = p[id], x0 = x[id];
            const T d1 = Dinv[id + NXY], r1 = r[id + NXY], p1 = p[id + NXY], x1 = x[id + NXY];
            finish(k, id, v0, d0, r0, p0, x0);
            finish(k + 1, id + NXY, v1, d1, r1, p1, x1);
        }
        if (k < k1) {
            T v0[8];
            nx.load(g, E, k, v0);
            finish(k, id, v0, Dinv[id], r[id], p[id], x[id]);
        }
    }
    double v[2];
    v[0] = block_sum_t(rzp);
    v[1] = block_sum_t(rrp);
    const unsigned nblk = gridDim.x * gridDim.y * gridDim.z;
    if (!publish_and_ticket(s, part + stride, v, 2, stride, nblk)) return;
    const double rz = last_cta_sum(part + stride, (int)nblk);
    const double rr = last_cta_sum(part + 2 * (size_t)stride, (int)nblk);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        s->ticket = 0;
        s->rr = rr;
        s->rz_new = rz;
        s->iters += 1;
        if (!isfinite(rz) || !isfinite(rr)) { s->status = ST_NAN; s->done = 1; }
        else if (rr <= s->tol2 * s->bb || s->iters >= s->max_iter) s->done = 1;
        s->beta = rz / s->rz;
        s->rz = rz;
    }
}

// ---------------------------------------------------------------------------
// Fused Jacobi-BiCGStab iteration over the two-pass apply (heat operator),
// five launches per iteration instead of thirteen:
//   cell A: ph = Dinv (r + beta (p - omega v)) at the cell's nodes, E = A_e ph
//           (heat_plane_kernel with the BiDirP input)
//   node A: p = r + beta (p - omega v) (the same formula), v = A ph;
//           last CTA: alpha = rho / rh.v
//   cell B: sh = Dinv (r - alpha v), E = A_e sh (heat_plane_kernel, BiDirS)
//   node B: t = A sh; last CTA: omega = t.s / t.t
//   update: x += alpha Dinv p + omega Dinv s, r = s - omega t with
//           s = r - alpha v; last CTA: convergence, beta, rho
// The lumped injection-well term of the heat operator (dt d_i on the
// diagonal of well nodes) is added in the node passes from a dense per-node
// array wd (null when there are no wells).  Dirichlet rows are identity rows:
// the node passes return the input there, as the plain apply does.
// Partial slots: 0 = rh.v; 1, 2 = t.s, t.t; 3, 4 = rh.r, r.r.
// ---------------------------------------------------------------------------
template <typename T>
struct BiDirP {   // ph = Dinv (r + beta (p - omega v))
    const T* r;
    const T* p;
    const T* v;
    const T* Dinv;
    T beta, omega;
    __device__ __forceinline__ void init(const Scal* s) { beta = (T)s->beta; omega = (T)s->omega; }
    __device__ __forceinline__ T val(int id) const { return fma(beta, fma(-omega, ldro(v + id), ldro(p + id)), ldro(r + id)); }
    __device__ __forceinline__ T operator()(int id) const { return ldro(Dinv + id) * val(id); }
};
template <typename T>
struct BiDirS {   // sh = Dinv (r - alpha v)
    const T* r;
    const T* v;
    const T* Dinv;
    T alpha;
    __device__ __forceinline__ void init(const Scal* s) { alpha = (T)s->alpha; }
    __device__ __forceinline__ T operator()(int id) const { return ldro(Dinv + id) * fma(-alpha, ldro(v + id), ldro(r + id)); }
};

// node A: p, v = A ph, partials of rh.v
template <int P, typename T>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 12 : 1) fbi_node_a_kernel(const Grid g, const T* __restrict__ E, const T* __restrict__ r,
                                                         T* __restrict__ p, T* __restrict__ v, const T* __restrict__ Dinv,
                                                         const T* __restrict__ rh, const T* __restrict__ wd, const T dt,
                                                         const int klen, Scal* s, double* __restrict__ part) {
    if (s->done) return;
    const T beta = (T)s->beta, omega = (T)s->omega;
    const int NXY = g.Nx * g.Ny;
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    T rv = T(0);
    if (m < NXY) {
        const NodeXY<P> nx(g, m % g.Nx, m / g.Nx);
        const int k0 = blockIdx.y * klen, k1 = min(k0 + klen, g.Nz);
        auto finish = [&](int k, int id, const T (&e)[8]) {
            const bool d = nx.dir || ((g.dmask & 16) && k == 0) || ((g.dmask & 32) && k == g.Nz - 1);
            const T pn = fma(beta, fma(-omega, v[id], p[id]), r[id]);
            const T ph = Dinv[id] * pn;
            T vn = ((e[0] + e[1]) + (e[2] + e[3])) + ((e[4] + e[5]) + (e[6] + e[7]));
            if (wd) vn += dt * wd[id] * ph;
            if (d) vn = ph;
            p[id] = pn;
            v[id] = vn;
            rv = fma(rh[id], vn, rv);
        };
        int k = k0, id = m + NXY * k0;
        for (; k + 1 < k1; k += 2, id += 2 * NXY) {
            T e0[8], e1[8];
            nx.load(g, E, k, e0);
            nx.load(g, E, k + 1, e1);
            finish(k, id, e0);
            finish(k + 1, id + NXY, e1);
        }
        if (k < k1) {
            T e0[8];
            nx.load(g, E, k, e0);
            finish(k, id, e0);
        }
    }
    const double tot = block_sum_t(rv);
    const unsigned nblk = gridDim.x * gridDim.y;
    if (!publish_and_ticket(s, part, &tot, 1, 0, nblk)) return;
    const double a = last_cta_sum(part, (int)nblk);
    if (threadIdx.x == 0) {
        s->ticket = 0;
        s->rv = a;
        if (a == 0.0 || !isfinite(a)) { s->status = ST_BREAKDOWN; s->done = 1; }
        else s->alpha = s->rho / a;
    }
}

// node B: t = A sh, partials of t.s and t.t
template <int P, typename T>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 12 : 1) fbi_node_b_kernel(const Grid g, const T* __restrict__ E, const T* __restrict__ r,
                                                         const T* __restrict__ v, T* __restrict__ t,
                                                         const T* __restrict__ Dinv, const T* __restrict__ wd,
                                                         const T dt, const int klen, Scal* s,
                                                         double* __restrict__ part, const int stride) {
    if (s->done) return;
    const T alpha = (T)s->alpha;
    const int NXY = g.Nx * g.Ny;
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    T ts = T(0), tt = T(0);
    if (m < NXY) {
        const NodeXY<P> nx(g, m % g.Nx, m / g.Nx);
        const int k0 = blockIdx.y * klen, k1 = min(k0 + klen, g.Nz);
        auto finish = [&](int k, int id, const T (&e)[8]) {
            const bool d = nx.dir || ((g.dmask & 16) && k == 0) || ((g.dmask & 32) && k == g.Nz - 1);
            const T si = fma(-alpha, v[id], r[id]);
            const T sh = Dinv[id] * si;
            T tn = ((e[0] + e[1]) + (e[2] + e[3])) + ((e[4] + e[5]) + (e[6] + e[7]));
            if (wd) tn += dt * wd[id] * sh;
            if (d) tn = sh;
            t[id] = tn;
            ts = fma(tn, si, ts);
            tt = fma(tn, tn, tt);
        };
        int k = k0, id = m + NXY * k0;
        for (; k + 1 < k1; k += 2, id += 2 * NXY) {
            T e0[8], e1[8];
            nx.load(g, E, k, e0);
            nx.load(g, E, k + 1, e1);
            finish(k, id, e0);
            finish(k + 1, id + NXY, e1);
        }
        if (k < k1) {
            T e0[8];
            nx.load(g, E, k, e0);
            finish(k, id, e0);
        }
    }
    double vals[2];
    vals[0] = block_sum_t(ts);
    vals[1] = block_sum_t(tt);
    const unsigned nblk = gridDim.x * gridDim.y;
    if (!publish_and_ticket(s, part + stride, vals, 2, stride, nblk)) return;
    const double a = last_cta_sum(part + stride, (int)nblk);
    const double b = last_cta_sum(part + 2 * (size_t)stride, (int)nblk);
    if (threadIdx.x == 0) {
        s->ticket = 0;
        s->ts = a;
        s->tt = b;
        s->omega = b == 0.0 ? 0.0 : a / b;   // s = 0 exactly: x += alpha ph is the solution
    }
}

// update: x, r; partials of rh.r and r.r; convergence and the next beta
template <typename T>
__global__ void __launch_bounds__(256) fbi_update_kernel(long long n, T* __restrict__ x, T* __restrict__ r,
                                                         const T* __restrict__ p, const T* __restrict__ v,
                                                         const T* __restrict__ t, const T* __restrict__ Dinv,
                                                         const T* __restrict__ rh, Scal* s,
                                                         double* __restrict__ part, const int stride) {
    if (s->done) return;
    const T alpha = (T)s->alpha, omega = (T)s->omega;
    T rhr = T(0), rr = T(0);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const T di = Dinv[i];
        const T si = fma(-alpha, v[i], r[i]);
        x[i] = fma(alpha, di * p[i], fma(omega, di * si, x[i]));
        const T ri = fma(-omega, t[i], si);
        r[i] = ri;
        rhr = fma(rh[i], ri, rhr);
        rr = fma(ri, ri, rr);
    }
    double vals[2];
    vals[0] = block_sum_t(rhr);
    vals[1] = block_sum_t(rr);
    const unsigned nblk = gridDim.x;
    if (!publish_and_ticket(s, part + 3 * (size_t)stride, vals, 2, stride, nblk)) return;
    const double a0 = last_cta_sum(part + 3 * (size_t)stride, (int)nblk);
    const double a1 = last_cta_sum(part + 4 * (size_t)stride, (int)nblk);
    if (threadIdx.x == 0) {
        s->ticket = 0;
        s->rr = a1;
        s->iters += 1;
        if (!isfinite(a0) || !isfinite(a1)) { s->status = ST_NAN; s->done = 1; }
        else if (a1 <= s->tol2 * s->bb || s->iters >= s->max_iter) s->done = 1;
        else if (a0 == 0.0 || s->omega == 0.0) { s->status = ST_BREAKDOWN; s->done = 1; }
        else {
            s->beta = (a0 / s->rho) * (s->alpha / s->omega);
            s->rho = a0;
        }
    }
}

// ---------------------------------------------------------------------------
// Right-hand sides through the element buffer.  Cells without Dirichlet nodes
// need only the mass term (light kernel); the few cells with Dirichlet nodes
// take the full lifted element RHS (heavy kernel over an enumeration of the
// face slabs).  The node pass sums the contributions in a fixed order and
// emits through the operator (g_D on Dirichlet rows, the sum plus dt F
// elsewhere).
// ---------------------------------------------------------------------------
// Cells of the slab next to a Dirichlet face: candidate t enumerates face 0's
// slab, then face 1's, ...; a cell in several slabs belongs to the first of
// them whose face is Dirichlet, so each boundary cell is done exactly once.
__device__ __forceinline__ bool face_cell(const Grid& g, long long t, int* cx, int* cy, int* cz) {
    const int dims[3] = {g.ncx, g.ncy, g.ncz};
    for (int f = 0; f < 6; ++f) {
        const int ax = f >> 1, u = ax == 0 ? 1 : 0, v = ax == 2 ? 1 : 2;
        const long long sz = (long long)dims[u] * dims[v];
        if (t >= sz) { t -= sz; continue; }
        if (!((g.dmask >> f) & 1)) return false;
        int c3[3];
        c3[ax] = (f & 1) ? dims[ax] - 1 : 0;
        c3[u] = (int)(t % dims[u]);
        c3[v] = (int)(t / dims[u]);
        for (int f2 = 0; f2 < f; ++f2) {
            const int ax2 = f2 >> 1;
            if (((g.dmask >> f2) & 1) && c3[ax2] == ((f2 & 1) ? dims[ax2] - 1 : 0)) return false;
        }
        *cx = c3[0]; *cy = c3[1]; *cz = c3[2];
        return true;
    }
    return false;
}

template <int P, typename T, class Op, typename ET = T>
__global__ void __launch_bounds__(128) rhs_boundary_kernel(const Grid g, const Op op, ET* __restrict__ E,
                                                           const long long n_cand) {
    constexpr int n = P + 1, NL = n * n * n;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    int cx, cy, cz;
    if (t >= n_cand || !face_cell(g, t, &cx, &cy, &cz)) return;
    const int nc = (int)g.nc;
    const int c = cx + g.ncx * (cy + g.ncy * cz);
    T res[NL];
    op.cell(g, cx, cy, cz, c, res);
#pragma unroll
    for (int l = 0; l < NL; ++l) E[l * nc + c] = cvt<ET>(res[l]);
}

// Mass-only right-hand side of the cells without Dirichlet nodes in
// float-float arithmetic: scale (G^T)^3 G^3 u_old with u_old split from FP64
// and scale S_s (head) or the cell's c_T (heat); cells with Dirichlet nodes
// are left to rhs_boundary_kernel.
template <int P>
__global__ void __launch_bounds__(128) rhs_interior_df_kernel(const Grid g, const Elem<df64> e,
                                                              const double* __restrict__ x,
                                                              const double* __restrict__ scale_c, const df64 scale_u,
                                                              df64* __restrict__ E, const int zlen) {
    constexpr int n = P + 1, NL = n * n * n;
    const int cx = blockIdx.x * blockDim.x + threadIdx.x;
    const int cy = blockIdx.y * blockDim.y + threadIdx.y;
    if (cx >= g.ncx || cy >= g.ncy) return;
    const int cz0 = blockIdx.z * zlen, cz1 = min(cz0 + zlen, g.ncz);
    const int nc = (int)g.nc, layer = g.ncx * g.ncy;
    const int NX = g.Nx, NXY = g.Nx * g.Ny;
    for (int cz = cz0; cz < cz1; ++cz) {
        if (cell_touches_dir(g, cx, cy, cz)) continue;
        const int c = cx + g.ncx * cy + layer * cz;
        const int base = P * cx + NX * P * cy + NXY * P * cz;
        df64 u[NL];
#pragma unroll
        for (int c2 = 0; c2 < n; ++c2)
#pragma unroll
            for (int b = 0; b < n; ++b)
#pragma unroll
                for (int a = 0; a < n; ++a) u[a + n * (b + n * c2)] = df_from(ldro(x + base + NX * b + NXY * c2 + a));
        sweep<n, 0, false>(u, e.G[0]);
        sweep<n, 1, false>(u, e.G[1]);
        sweep<n, 2, false>(u, e.G[2]);
        df64 sc = scale_c ? df_from(ldro(scale_c + c)) : scale_u;
        if (g.geo64) sc = sc * df_from(ldro(g.geo64 + c));   // graded mesh: times the cell volume
#pragma unroll
        for (int l = 0; l < NL; ++l) u[l] = u[l] * sc;
        sweep<n, 2, true>(u, e.G[2]);
        sweep<n, 1, true>(u, e.G[1]);
        sweep<n, 0, true>(u, e.G[0]);
#pragma unroll
        for (int l = 0; l < NL; ++l) E[l * nc + c] = u[l];
    }
}

// node pass of the right-hand side from float-float contributions
template <int P, class Op>
__global__ void __launch_bounds__(128) node_emit_df_kernel(const Grid g, const df64* __restrict__ E, const Op op,
                                                           const int klen) {
    const int NXY = g.Nx * g.Ny;
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= NXY) return;
    const int i = m % g.Nx, j = m / g.Nx;
    const NodeXY<P> nx(g, i, j);
    const int k0 = blockIdx.y * klen, k1 = min(k0 + klen, g.Nz);
    double dot = 0.0;
    for (int k = k0; k < k1; ++k) {
        df64 v[8];
        nx.load(g, E, k, v);
        const df64 sum = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
        op.emit(g, i, j, k, df_to(sum), dot);
    }
}


// ---------------------------------------------------------------------------
// Outer residual of the mixed form in float-float arithmetic: the element pass
// splits the FP64 iterate into float pairs (Dirichlet nodes zero) and applies
// the element operator in float-float; the node pass sums the contributions
// in float-float, returns to FP64 for r = b - A x (and the lumped well term),
// and writes (float) r for the next inner solve and partial sums of r.r and
// b.b.  The element buffer is the FP64 one, read as float pairs.
// ---------------------------------------------------------------------------
template <int P, class Op>
__global__ void __launch_bounds__(128) df_cell_kernel(const Grid g, const Op op, const df64* __restrict__ x,
                                                      df64* __restrict__ E, const int zlen) {
    constexpr int n = P + 1, NL = n * n * n;
    const int cx = blockIdx.x * blockDim.x + threadIdx.x;
    const int cy = blockIdx.y * blockDim.y + threadIdx.y;
    if (cx >= g.ncx || cy >= g.ncy) return;
    const int cz0 = blockIdx.z * zlen, cz1 = min(cz0 + zlen, g.ncz);
    const int nc = (int)g.nc, layer = g.ncx * g.ncy;
    const int NX = g.Nx, NXY = g.Nx * g.Ny;
    const bool edge_xy = g.dmask != 0 && (cx == 0 || cx == g.ncx - 1 || cy == 0 || cy == g.ncy - 1);
    int base = P * cx + NX * P * cy + NXY * P * cz0;
    int c = cx + g.ncx * cy + layer * cz0;
    for (int cz = cz0; cz < cz1; ++cz, base += NXY * P, c += layer) {
        df64 u[NL];
#pragma unroll
        for (int c2 = 0; c2 < n; ++c2)
#pragma unroll
            for (int b = 0; b < n; ++b)
#pragma unroll
                for (int a = 0; a < n; ++a) u[a + n * (b + n * c2)] = ldg_any<df64>(x + base + NX * b + NXY * c2 + a);
        if (edge_xy || (g.dmask & 48 && (cz == 0 || cz == g.ncz - 1))) {
#pragma unroll
            for (int c2 = 0; c2 < n; ++c2)
#pragma unroll
                for (int b = 0; b < n; ++b)
#pragma unroll
                    for (int a = 0; a < n; ++a)
                        if (on_dir(g, P * cx + a, P * cy + b, P * cz + c2)) u[a + n * (b + n * c2)] = df64(0);
        }
        df64 res[NL];
        op.compute(u, c, res);
#pragma unroll
        for (int l = 0; l < NL; ++l) E[l * nc + c] = res[l];
    }
}

template <int P>
__global__ void __launch_bounds__(128) df_resid_node_kernel(const Grid g, const df64* __restrict__ E,
                                                            const double* __restrict__ x,
                                                            const double* __restrict__ b,
                                                            const double* __restrict__ wd, const double dt,
                                                            float* __restrict__ r32, double* __restrict__ part,
                                                            const int stride, const int klen) {
    const int NXY = g.Nx * g.Ny;
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    double rr = 0.0, bb = 0.0;
    if (m < NXY) {
        const NodeXY<P> nx(g, m % g.Nx, m / g.Nx);
        const int k0 = blockIdx.y * klen, k1 = min(k0 + klen, g.Nz);
        for (int k = k0; k < k1; ++k) {
            const int id = m + NXY * k;
            df64 v[8];
            nx.load(g, E, k, v);
            const df64 sum = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
            const bool d = nx.dir || ((g.dmask & 16) && k == 0) || ((g.dmask & 32) && k == g.Nz - 1);
            const double xi = x[id];
            double y = d ? xi : df_to(sum);
            if (wd && !d) y = fma(dt * wd[id], xi, y);
            const double bi = b[id];
            const double ri = bi - y;
            r32[id] = (float)ri;
            rr = fma(ri, ri, rr);
            bb = fma(bi, bi, bb);
        }
    }
    const double a0 = block_sum(rr);
    const double a1 = block_sum(bb);
    if (threadIdx.x == 0) {
        const int blk = blockIdx.x + gridDim.x * blockIdx.y;
        part[blk] = a0;
        part[(size_t)stride + blk] = a1;
    }
}

// ---------------------------------------------------------------------------
// Heat element pass with one thread per Gauss plane: a CTA of 32 x (P+1)
// threads takes 32 cells of a row and marches them in z.  Thread (tx, qz)
// forms the operator input at node layer qz of its cell (nv(id), Dirichlet
// nodes zero) in shared memory, computes the contribution of plane qz
// (HeatOp::plane) into shared memory, and finally sums the planes'
// contributions to node layer qz in a fixed order and writes them to E.
// The three planes split the work and the registers of one cell.
// ---------------------------------------------------------------------------
template <typename T>
struct LoadNodes {   // plain operator input
    const T* x;
    __device__ __forceinline__ void init(const Scal*) {}
    __device__ __forceinline__ T operator()(int id) const { return ldro(x + id); }
};
struct LoadSplit {   // FP64 input split into float pairs
    const double* x;
    __device__ __forceinline__ void init(const Scal*) {}
    __device__ __forceinline__ df64 operator()(int id) const { return df_from(ldro(x + id)); }
};

template <int P, typename T, class Op, class NV, bool HQ>
__global__ void __launch_bounds__(32 * (P + 1)) heat_plane_kernel(const Grid g, const Op op, NV nv,
                                                                  const T* __restrict__ hq, T* __restrict__ E,
                                                                  const int zlen, const Scal* s) {
    if (s && s->done) return;
    if (s) nv.init(s);
    constexpr int n = P + 1, NL = n * n * n;
    __shared__ T su[32][NL];
    __shared__ T sh[HQ ? 32 : 1][NL];
    __shared__ T sp[n][32][NL];
    const int tx = threadIdx.x, qz = threadIdx.y;
    const int cx = blockIdx.x * 32 + tx, cy = blockIdx.y;
    const bool valid = cx < g.ncx;
    const int cz0 = blockIdx.z * zlen, cz1 = min(cz0 + zlen, g.ncz);
    const int nc = (int)g.nc, layer = g.ncx * g.ncy;
    const int NX = g.Nx, NXY = g.Nx * g.Ny;
    const bool edge_xy = g.dmask != 0 && (cx == 0 || cx == g.ncx - 1 || cy == 0 || cy == g.ncy - 1);
    int base = P * cx + NX * P * cy + NXY * P * cz0;
    int c = cx + g.ncx * cy + layer * cz0;
    for (int cz = cz0; cz < cz1; ++cz, base += NXY * P, c += layer) {
        if (valid) {
            const bool chk = edge_xy || ((g.dmask & 48) && (cz == 0 || cz == g.ncz - 1));
#pragma unroll
            for (int b = 0; b < n; ++b)
#pragma unroll
                for (int a = 0; a < n; ++a) {
                    const int id = base + NX * b + NXY * qz + a;
                    T u = nv(id);
                    if (chk && on_dir(g, P * cx + a, P * cy + b, P * cz + qz)) u = T(0);
                    su[tx][a + n * (b + n * qz)] = u;
                    if constexpr (HQ) sh[tx][a + n * (b + n * qz)] = ldg_any(hq + id);
                }
        }
        __syncthreads();
        if (valid) op.template plane<HQ>(&su[tx][0], HQ ? &sh[HQ ? tx : 0][0] : nullptr, c, nc, qz, &sp[qz][tx][0]);
        __syncthreads();
        if (valid) {
#pragma unroll
            for (int ba = 0; ba < n * n; ++ba) {
                const int l = ba + n * n * qz;
                T v = sp[0][tx][l];
#pragma unroll
                for (int q = 1; q < n; ++q) v = v + sp[q][tx][l];
                E[l * nc + c] = v;
            }
        }
    }
}

// grid of heat_plane_kernel: 32-cell row segments x rows x a split of the layers
template <auto Kernel>
int resident_per_sm_threads(int threads) {
    static const int r = [threads] {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, Kernel, threads, 0) != cudaSuccess || v < 1) v = 1;
        return v;
    }();
    return r;
}

// ---------------------------------------------------------------------------
// Other per-cell kernels
// ---------------------------------------------------------------------------
// q = -K_c grad h at the Gauss points; qs[(d*NQ + q)*nc + c]
template <int P>
__global__ void darcy_qp_kernel(const Grid g, const double* __restrict__ h,
                                const double* __restrict__ K, const Elem<double> e,
                                double* __restrict__ qs64, float* __restrict__ qs32) {
    constexpr int n = P + 1, NL = n * n * n, NQ = NL;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < g.nc;
         c += (long long)gridDim.x * blockDim.x) {
        const int cx = (int)(c % g.ncx), cy = (int)((c / g.ncx) % g.ncy), cz = (int)(c / ((long long)g.ncx * g.ncy));
        double u[NL];
        gather<P, double>(g, h, cx, cy, cz, false, u);
        const double Kc = K[c];
        double ih[3] = {e.invH[0], e.invH[1], e.invH[2]};
        if (g.geo64)
            for (int d = 0; d < 3; ++d) ih[d] = g.geo64[(d + 1) * g.nc + c];
        // gradient at the Gauss points by sum factorisation: z, then y, then x
        double zB[NQ], zD[NQ];   // [qz][b][a]
#pragma unroll
        for (int qz = 0; qz < n; ++qz)
#pragma unroll
            for (int ba = 0; ba < n * n; ++ba) {
                double sb = 0, sd = 0;
#pragma unroll
                for (int c2 = 0; c2 < n; ++c2) {
                    sb = fma(e.B[qz][c2], u[ba + n * n * c2], sb);
                    sd = fma(e.D[qz][c2], u[ba + n * n * c2], sd);
                }
                zB[qz * n * n + ba] = sb;
                zD[qz * n * n + ba] = sd;
            }
#pragma unroll
        for (int qz = 0; qz < n; ++qz)
#pragma unroll
            for (int qy = 0; qy < n; ++qy) {
                double yBB[n], yDB[n], yBD[n];
#pragma unroll
                for (int a = 0; a < n; ++a) {
                    double v0 = 0, v1 = 0, v2 = 0;
#pragma unroll
                    for (int b = 0; b < n; ++b) {
                        v0 = fma(e.B[qy][b], zB[qz * n * n + a + n * b], v0);
                        v1 = fma(e.D[qy][b], zB[qz * n * n + a + n * b], v1);
                        v2 = fma(e.B[qy][b], zD[qz * n * n + a + n * b], v2);
                    }
                    yBB[a] = v0; yDB[a] = v1; yBD[a] = v2;
                }
#pragma unroll
                for (int qx = 0; qx < n; ++qx) {
                    double gx = 0, gy = 0, gz = 0;
#pragma unroll
                    for (int a = 0; a < n; ++a) {
                        gx = fma(e.D[qx][a], yBB[a], gx);
                        gy = fma(e.B[qx][a], yDB[a], gy);
                        gz = fma(e.B[qx][a], yBD[a], gz);
                    }
                    const int qi = qx + n * (qy + n * qz);
                    const double q0 = -Kc * gx * ih[0];
                    const double q1 = -Kc * gy * ih[1];
                    const double q2 = -Kc * gz * ih[2];
                    qs64[(0 * NQ + qi) * g.nc + c] = q0;
                    qs64[(1 * NQ + qi) * g.nc + c] = q1;
                    qs64[(2 * NQ + qi) * g.nc + c] = q2;
                    qs32[(0 * NQ + qi) * g.nc + c] = (float)q0;
                    qs32[(1 * NQ + qi) * g.nc + c] = (float)q1;
                    qs32[(2 * NQ + qi) * g.nc + c] = (float)q2;
                }
            }
    }
}

struct CentreBasis { double v[3], d[3]; };

template <int P>
__global__ void cell_flux_kernel(const Grid g, const double* __restrict__ h,
                                 const double* __restrict__ K, const CentreBasis cb,
                                 const double invH, const int comp, double* __restrict__ out) {
    constexpr int n = P + 1, NL = n * n * n;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < g.nc;
         c += (long long)gridDim.x * blockDim.x) {
        const int cx = (int)(c % g.ncx), cy = (int)((c / g.ncx) % g.ncy), cz = (int)(c / ((long long)g.ncx * g.ncy));
        double u[NL];
        gather<P, double>(g, h, cx, cy, cz, false, u);
        double s = 0;
#pragma unroll
        for (int c2 = 0; c2 < n; ++c2)
#pragma unroll
            for (int b = 0; b < n; ++b)
#pragma unroll
                for (int a = 0; a < n; ++a) {
                    const double fa = comp == 0 ? cb.d[a] : cb.v[a];
                    const double fb = comp == 1 ? cb.d[b] : cb.v[b];
                    const double fc = comp == 2 ? cb.d[c2] : cb.v[c2];
                    s += fa * fb * fc * u[a + n * (b + n * c2)];
                }
        out[c] = -K[c] * s * (g.geo64 ? g.geo64[(comp + 1) * g.nc + c] : invH);
    }
}

template <typename T>
__global__ void well_apply_kernel(int n, const int* __restrict__ node, const double* __restrict__ d,
                                  T dt, const T* __restrict__ x, T* __restrict__ y,
                                  const Scal* __restrict__ sc) {
    if (sc && sc->done) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const int id = node[i];
        y[id] += dt * (T)d[i] * x[id];
    }
}

template <typename T>
__global__ void well_diag_kernel(int n, const int* __restrict__ node, const double* __restrict__ d,
                                 double dt, T* __restrict__ D) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) D[node[i]] += (T)(dt * d[i]);
}

__global__ void pile_load_kernel(int n_nodes, const int* __restrict__ node, const int* __restrict__ off,
                                 const int* __restrict__ src, const double* __restrict__ w,
                                 const ht_line_src* __restrict__ piles, double t,
                                 const double* __restrict__ Fbase, double* __restrict__ F) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_nodes) {
        const int id = node[i];
        double s = Fbase[id];
        for (int e = off[i]; e < off[i + 1]; ++e) {
            const ht_line_src& pl = piles[src[e]];
            const double a = pl.mean + pl.amp * sin(2.0 * 3.141592653589793 * t / pl.period + pl.phase);
            s += a * w[e];
        }
        F[id] = s;
    }
}

__global__ void add_kernel(long long n, const double* __restrict__ a, const double* __restrict__ b,
                           double* __restrict__ out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = a[i] + (b ? b[i] : 0.0);
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
namespace {

constexpr int kCXM = 16, kCYM = 16;

Grid field_grid(const ht_ctx* c, int field) {
    Grid g = c->grid;
    g.dmask = c->dmask[field];
    return g;
}

template <int P>
void tile_dims(const ht_ctx* c, dim3* grid, int* ZC) {
    using S = TileShape<P, kCXM, kCYM>;
    const Grid& g = c->grid;
    const int tx = (g.Nx + S::TX - 1) / S::TX, ty = (g.Ny + S::TY - 1) / S::TY;
    const int target = 2 * (c->num_sms > 0 ? c->num_sms : 148);
    int chunks = (target + tx * ty - 1) / (tx * ty);
    if (c->opts.z_chunks > 0) chunks = c->opts.z_chunks;
    chunks = chunks < 1 ? 1 : (chunks > g.ncz ? g.ncz : chunks);
    int zc = (g.ncz + chunks - 1) / chunks;
    chunks = (g.ncz + zc - 1) / zc;
    *grid = dim3(tx, ty, chunks);
    *ZC = zc;
}

template <int P, typename T, class Op>
int launch_tile(ht_ctx* c, const Grid& g, const Op& op, double* dot_part, int* n_part,
                const Scal* sc = nullptr) {
    dim3 grid;
    int ZC;
    tile_dims<P>(c, &grid, &ZC);
    constexpr int n = P + 1, NL = n * n * n;
    const size_t smem = (size_t)kCXM * kCYM * NL * sizeof(T);
    auto kern = tile_kernel<P, T, kCXM, kCYM, Op>;
    static bool attr_done = false;   // per instantiation
    if (!attr_done) {
        HT_CUDA(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr_done = true;
    }
    kern<<<grid, kCXM * kCYM, smem, c->stream>>>(g, op, ZC, dot_part, sc); ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    if (n_part) *n_part = (int)(grid.x * grid.y * grid.z);
    return HT_OK;
}

template <int P, typename T, class Op>
int launch_apply_staged(ht_ctx* c, const Grid& g, const Op& op, const T* x, T* y, double* dot_part,
                        int* n_part, const Scal* sc) {
    dim3 grid;
    int ZC;
    tile_dims<P>(c, &grid, &ZC);
    const size_t smem = ApplySmem<P, kCXM, kCYM, T>::bytes;
    auto kern = apply_kernel<P, T, kCXM, kCYM, Op>;
    static bool attr_done = false;   // per instantiation
    if (!attr_done) {
        HT_CUDA(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr_done = true;
    }
    kern<<<grid, kCXM * kCYM, smem, c->stream>>>(g, op, ZC, x, y, dot_part, sc); ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    if (n_part) *n_part = (int)(grid.x * grid.y * grid.z);
    return HT_OK;
}

template <typename T>
T* elem_buffer(ht_ctx* c);
template <>
double* elem_buffer<double>(ht_ctx* c) { return c->E64 ? c->E64 + kElemPad : nullptr; }
template <>
float* elem_buffer<float>(ht_ctx* c) { return c->E32 ? c->E32 + kElemPad : nullptr; }

// resident 128-thread CTAs of a kernel per SM (queried once per kernel)
template <auto Kernel>
int resident_per_sm() {
    static const int n = [] {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, Kernel, 128, 0) != cudaSuccess || v < 1) v = 1;
        return v;
    }();
    return n;
}

// Split of a marching range of n layers over `cols` thread columns: the split
// z minimises (waves of resident CTAs) x (layers per CTA + 1), the "+ 1" being
// the start-up of a CTA; ties go to fewer CTAs.  zmax bounds the split.
int pick_split(int n, int cols, int resident, int zmax) {
    int best = 1;
    long long best_cost = -1;
    for (int z = 1; z <= n && z <= zmax; ++z) {
        const int len = (n + z - 1) / z;
        if (z > 1 && (n + len - 1) / len != z) continue;  // same as a smaller split
        const long long waves = ((long long)cols * z + resident - 1) / resident;
        const long long cost = waves * (len + 1);
        if (best_cost < 0 || cost < best_cost) { best_cost = cost; best = z; }
    }
    return best;
}

// cell-pass grid of the two-pass kernels, shared by the apply and the fused
// CG: (32 x 4) cell columns marching in z
void cell_pass_dims(const ht_ctx* c, const Grid& g, int cell_per_sm, dim3* grid, int* zlen) {
    const int sms = c->num_sms > 0 ? c->num_sms : 148;
    const int gx = (g.ncx + 31) / 32, gy = (g.ncy + 3) / 4;
    int zs = pick_split(g.ncz, gx * gy, cell_per_sm * sms, c->part_stride / (gx * gy));
    *zlen = (g.ncz + zs - 1) / zs;
    zs = (g.ncz + *zlen - 1) / *zlen;
    *grid = dim3(gx, gy, zs);
}

// grid of heat_plane_kernel: 32-cell row segments x rows x a split of the layers
void plane_pass_dims(const ht_ctx* c, const Grid& g, int cta_per_sm, dim3* grid, int* zlen) {
    const int sms = c->num_sms > 0 ? c->num_sms : 148;
    const int gx = (g.ncx + 31) / 32;
    int zs = pick_split(g.ncz, gx * g.ncy, cta_per_sm * sms, g.ncz);
    *zlen = (g.ncz + zs - 1) / zs;
    zs = (g.ncz + *zlen - 1) / *zlen;
    *grid = dim3(gx, g.ncy, zs);
}

// launch of the element pass of a heat operator with input functor nv
template <int P, typename T, class Op, class NV>
int launch_heat_planes(ht_ctx* c, const Grid& g, const Op& op, const NV& nv, T* E, const Scal* sc,
                       const T* hq = nullptr) {
    constexpr int threads = 32 * (P + 1);
    dim3 grid;
    int zlen;
    if constexpr (sizeof(T) == 4) {   // the head-formed velocity is an FP32-operator feature
        if (hq) {
            plane_pass_dims(c, g, resident_per_sm_threads<heat_plane_kernel<P, T, Op, NV, true>>(threads), &grid,
                            &zlen);
            heat_plane_kernel<P, T, Op, NV, true><<<grid, dim3(32, P + 1), 0, c->stream>>>(g, op, nv, hq, E, zlen,
                                                                                          sc);
            ++c->n_launch;
            HT_CUDA(c, cudaGetLastError());
            return HT_OK;
        }
    }
    plane_pass_dims(c, g, resident_per_sm_threads<heat_plane_kernel<P, T, Op, NV, false>>(threads), &grid, &zlen);
    heat_plane_kernel<P, T, Op, NV, false><<<grid, dim3(32, P + 1), 0, c->stream>>>(g, op, nv, hq, E, zlen, sc);
    ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    return HT_OK;
}

// node-pass grid: 128-node runs of a layer x a split of the layers; the block
// count bounds the partial sums
void layer_node_dims(const ht_ctx* c, const Grid& g, int node_per_sm, dim3* grid, int* klen) {
    const int sms = c->num_sms > 0 ? c->num_sms : 148;
    const int runs = (g.Nx * g.Ny + 127) / 128;
    int ks = pick_split(g.Nz, runs, node_per_sm * sms, c->part_stride / runs);
    *klen = (g.Nz + ks - 1) / ks;
    ks = (g.Nz + *klen - 1) / *klen;
    *grid = dim3(runs, ks);
}

template <int P, typename T, class Op>
int launch_apply_two_pass(ht_ctx* c, const Grid& g, const Op& op, const T* x, T* y, double* dot_part,
                          int* n_part, const Scal* sc) {
    T* E = elem_buffer<T>(c);
    dim3 ngrid;
    int klen;
    layer_node_dims(c, g, resident_per_sm<node_pass_kernel<P, T>>(), &ngrid, &klen);
    const int nb = (int)(ngrid.x * ngrid.y);
    if (dot_part && nb > c->part_stride) return fail(c, HT_EINVAL, "too many partial sums");
    if constexpr (Op::kPlanes) {
        // FP32: the velocity is formed from the FP32 head, as in the fused BiCGStab
        Op opq = op;
        const T* hq = sizeof(T) == 4 ? (const T*)c->h32 : nullptr;
        if (hq) opq.Kq = (const T*)c->K32;
        HT_TRY((launch_heat_planes<P, T>(c, g, opq, LoadNodes<T>{x}, E, sc, hq)));
    } else {
        dim3 cgrid;
        int zlen;
        cell_pass_dims(c, g, resident_per_sm<cell_pass_kernel<P, T, Op>>(), &cgrid, &zlen);
        cell_pass_kernel<P, T, Op><<<cgrid, dim3(32, 4), 0, c->stream>>>(g, op, x, E, zlen, sc); ++c->n_launch;
        HT_CUDA(c, cudaGetLastError());
    }
    node_pass_kernel<P, T><<<ngrid, 128, 0, c->stream>>>(g, E, x, y, klen, dot_part, sc); ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    if (n_part) *n_part = nb;
    return HT_OK;
}

template <typename T>
bool use_two_pass(const ht_ctx* c) {
    const int v = c->opts.apply_variant;
    if (v == HT_APPLY_TILED) return false;
    if (!elem_buffer<T>(const_cast<ht_ctx*>(c))) return false;
    if (v == HT_APPLY_TWO_PASS) return true;
    return sizeof(T) == 4;   // automatic choice: two-pass for FP32, tiled for FP64
}

template <typename T>
const Elem<T>& elem_of(const ht_ctx* c);
template <>
const Elem<double>& elem_of<double>(const ht_ctx* c) { return c->e64; }
template <>
const Elem<float>& elem_of<float>(const ht_ctx* c) { return c->e32; }

// the per-cell geometry of a graded mesh in the operator's storage type
template <class Op>
void set_geo(Op& op, const ht_ctx* c) {
    using S = std::remove_const_t<std::remove_pointer_t<decltype(op.geo)>>;
    if constexpr (std::is_same<S, float>::value) op.geo = c->geo32;
    else op.geo = c->geo64;
    op.gnc = c->grid.nc;
}

template <int P, typename T>
int fused_cg_iteration_P(ht_ctx* c, T dt, T* x, T* r, const T* Dinv, T* p, Scal* sc, int first) {
    using Op = HeadOp<P, T, MODE_APPLY>;
    const Grid g = field_grid(c, HT_HEAD);
    Op op{};
    op.K = sizeof(T) == 8 ? (const T*)c->K64 : (const T*)c->K32;
    op.alpha = (T)c->Ss;
    op.dt = dt;
    op.e = elem_of<T>(c);
    set_geo(op, c);
    T* E = elem_buffer<T>(c);
    dim3 cgrid, ngrid;
    int zlen, klen;
    cell_pass_dims(c, g, resident_per_sm<fcg_cell_kernel<P, T, Op>>(), &cgrid, &zlen);
    layer_node_dims(c, g, resident_per_sm<fcg_node_kernel<P, T>>(), &ngrid, &klen);
    if ((int)(cgrid.x * cgrid.y * cgrid.z) > c->part_stride || (int)(ngrid.x * ngrid.y) > c->part_stride)
        return fail(c, HT_EINVAL, "too many partial sums");
    fcg_cell_kernel<P, T, Op><<<cgrid, dim3(32, 4), 0, c->stream>>>(g, op, r, Dinv, p, E, zlen, sc, c->part, first);
    ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    fcg_node_kernel<P, T><<<ngrid, 128, 0, c->stream>>>(g, E, x, r, Dinv, p, klen, sc, c->part, c->part_stride,
                                                        first);
    ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    return HT_OK;
}

template <typename T>
const T* well_dense(const ht_ctx* c);
template <>
const double* well_dense<double>(const ht_ctx* c) { return c->wdn64; }
template <>
const float* well_dense<float>(const ht_ctx* c) { return c->wdn32; }

template <int P, typename T>
int fused_bicgstab_iteration_P(ht_ctx* c, T dt, T* x, T* r, const T* rh, T* p, T* v, T* t, const T* Dinv,
                               Scal* sc) {
    using Op = HeatOp<P, T, MODE_APPLY>;
    const Grid g = field_grid(c, HT_TEMP);
    const bool f64 = sizeof(T) == 8;
    Op op{};
    op.qs = f64 ? (const T*)c->qs64 : (const T*)c->qs32;
    op.cTc = f64 ? (const T*)c->cT64 : (const T*)c->cT32;
    op.lamc = f64 ? (const T*)c->lam64 : (const T*)c->lam32;
    op.cT_u = (T)c->cT_u; op.lam_u = (T)c->lam_u; op.dt = dt; op.cw = (T)c->cw;
    op.e = elem_of<T>(c);
    set_geo(op, c);
    op.g_nc = g.nc;
    T* E = elem_buffer<T>(c);
    const T* wd = well_dense<T>(c);
    dim3 na, nb;
    int ka, kb;
    layer_node_dims(c, g, resident_per_sm<fbi_node_a_kernel<P, T>>(), &na, &ka);
    layer_node_dims(c, g, resident_per_sm<fbi_node_b_kernel<P, T>>(), &nb, &kb);
    const int G = vec_grid(c);
    if ((int)(na.x * na.y) > c->part_stride || (int)(nb.x * nb.y) > c->part_stride || G > c->part_stride)
        return fail(c, HT_EINVAL, "too many partial sums");
    const int S = c->part_stride;
    // FP32: the velocity is formed from the FP32 head in the element pass
    const T* hq = f64 ? nullptr : (const T*)c->h32;
    if (hq) op.Kq = (const T*)c->K32;
    HT_TRY((launch_heat_planes<P, T>(c, g, op, BiDirP<T>{r, p, v, Dinv, T(0), T(0)}, E, sc, hq)));
    fbi_node_a_kernel<P, T><<<na, 128, 0, c->stream>>>(g, E, r, p, v, Dinv, rh, wd, dt, ka, sc, c->part); ++c->n_launch;
    HT_TRY((launch_heat_planes<P, T>(c, g, op, BiDirS<T>{r, v, Dinv, T(0)}, E, sc, hq)));
    fbi_node_b_kernel<P, T><<<nb, 128, 0, c->stream>>>(g, E, r, v, t, Dinv, wd, dt, kb, sc, c->part, S); ++c->n_launch;
    fbi_update_kernel<T><<<G, 256, 0, c->stream>>>(c->grid.nn, x, r, p, v, t, Dinv, rh, sc, c->part, S);
    ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    return HT_OK;
}

template <int P, typename T>
int apply_P(ht_ctx* c, int field, T dt, const T* x, T* y, double* dot_part, int* n_part,
            const Scal* sc) {
    const Grid g = field_grid(c, field);
    const bool f64 = sizeof(T) == 8;
    if (field == HT_HEAD) {
        HeadOp<P, T, MODE_APPLY> op{};
        op.x = x; op.y = y;
        op.K = f64 ? (const T*)c->K64 : (const T*)c->K32;
        op.alpha = (T)c->Ss; op.dt = dt; op.e = elem_of<T>(c);
        set_geo(op, c);
        if (use_two_pass<T>(c)) return launch_apply_two_pass<P, T>(c, g, op, x, y, dot_part, n_part, sc);
        return launch_apply_staged<P, T>(c, g, op, x, y, dot_part, n_part, sc);
    }
    HeatOp<P, T, MODE_APPLY> op{};
    op.x = x; op.y = y;
    op.qs = f64 ? (const T*)c->qs64 : (const T*)c->qs32;
    op.cTc = f64 ? (const T*)c->cT64 : (const T*)c->cT32;
    op.lamc = f64 ? (const T*)c->lam64 : (const T*)c->lam32;
    op.cT_u = (T)c->cT_u; op.lam_u = (T)c->lam_u; op.dt = dt; op.cw = (T)c->cw;
    op.e = elem_of<T>(c);
    set_geo(op, c);
    op.g_nc = g.nc;
    if (use_two_pass<T>(c)) return launch_apply_two_pass<P, T>(c, g, op, x, y, dot_part, n_part, sc);
    return launch_apply_staged<P, T>(c, g, op, x, y, dot_part, n_part, sc);
}

}  // namespace

// one fused CG iteration of the head system (see fcg_cell_kernel)
int fused_cg_iteration64(ht_ctx* c, double dt, double* x, double* r, const double* Dinv, double* p, Scal* sc,
                         int first) {
    return c->grid.P == 1 ? fused_cg_iteration_P<1, double>(c, dt, x, r, Dinv, p, sc, first)
                          : fused_cg_iteration_P<2, double>(c, dt, x, r, Dinv, p, sc, first);
}
int fused_cg_iteration32(ht_ctx* c, float dt, float* x, float* r, const float* Dinv, float* p, Scal* sc,
                         int first) {
    return c->grid.P == 1 ? fused_cg_iteration_P<1, float>(c, dt, x, r, Dinv, p, sc, first)
                          : fused_cg_iteration_P<2, float>(c, dt, x, r, Dinv, p, sc, first);
}
int launch_fbi_update32(ht_ctx* c, float* x, float* r, const float* p, const float* v, const float* t,
                        const float* Dinv, const float* rh, Scal* sc) {
    const int G = vec_grid(c);
    if (G > c->part_stride) return fail(c, HT_EINVAL, "too many partial sums");
    fbi_update_kernel<float><<<G, 256, 0, c->stream>>>(c->grid.nn, x, r, p, v, t, Dinv, rh, sc, c->part,
                                                        c->part_stride);
    ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    return HT_OK;
}

int fused_bicgstab_iteration64(ht_ctx* c, double dt, double* x, double* r, const double* rh, double* p, double* v,
                               double* t, const double* Dinv, Scal* sc) {
    return c->grid.P == 1 ? fused_bicgstab_iteration_P<1, double>(c, dt, x, r, rh, p, v, t, Dinv, sc)
                          : fused_bicgstab_iteration_P<2, double>(c, dt, x, r, rh, p, v, t, Dinv, sc);
}
int fused_bicgstab_iteration32(ht_ctx* c, float dt, float* x, float* r, const float* rh, float* p, float* v,
                               float* t, const float* Dinv, Scal* sc) {
    return c->grid.P == 1 ? fused_bicgstab_iteration_P<1, float>(c, dt, x, r, rh, p, v, t, Dinv, sc)
                          : fused_bicgstab_iteration_P<2, float>(c, dt, x, r, rh, p, v, t, Dinv, sc);
}
bool fused_cg_available(const ht_ctx* c, int fp32) {
    return fp32 ? use_two_pass<float>(c) : use_two_pass<double>(c);
}

int apply_tiles(const ht_ctx* c) {
    dim3 grid;
    int ZC;
    if (c->grid.P == 1) tile_dims<1>(c, &grid, &ZC);
    else tile_dims<2>(c, &grid, &ZC);
    return (int)(grid.x * grid.y * grid.z);
}

// ---- Dirichlet rows that change with time or lie inside the mesh ------------
// Seasonal faces and pile surfaces (Section 3.3) take their values at each
// step's t^{n+1}.  A pile-surface node off the Dirichlet faces is a Dirichlet
// row of the heat system like a face node: its row of A0 is the identity row
// and its column is removed (A0 = P A P + (I - P), P the projector on the
// free nodes).  The raw operator kernels treat the six faces only, so the
// heat operator launches below wrap them: the input with the interior rows
// zeroed (the columns removed), then those rows of the output set to the
// input (the identity rows); the diagonal is 1 there, and the lifted
// right-hand side takes A0 g of the interior values off the free rows.
namespace {

// face `face` at value v, except nodes on a Dirichlet face of higher index
// (on a shared edge the higher face wins)
__global__ void face_value_kernel(Grid g, int face, double v, double* __restrict__ gval) {
    const int axis = face / 2, side = face % 2;
    const int Nd[3] = {g.Nx, g.Ny, g.Nz};
    const int t1 = axis == 0 ? 1 : 0, t2 = axis == 2 ? 1 : 2;
    const long long n = (long long)Nd[t1] * Nd[t2];
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x) {
        int ijk[3];
        ijk[axis] = side ? Nd[axis] - 1 : 0;
        ijk[t1] = (int)(q % Nd[t1]);
        ijk[t2] = (int)(q / Nd[t1]);
        bool higher = false;
        for (int f2 = face + 1; f2 < 6; ++f2) {
            const int a2 = f2 / 2;
            if (((g.dmask >> f2) & 1) && ijk[a2] == ((f2 & 1) ? Nd[a2] - 1 : 0)) higher = true;
        }
        if (!higher) gval[ijk[0] + (long long)g.Nx * (ijk[1] + (long long)g.Ny * ijk[2])] = v;
    }
}

// pile surfaces: T_mean + T_amp sign(sin(2 pi t / period + phase)), sign(0) = +1
__global__ void pile_temp_kernel(int n, const long long* __restrict__ node, const int* __restrict__ pile,
                                 const double* __restrict__ prm, double t, double* __restrict__ gval) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double* pr = prm + 4 * pile[i];
    const double sn = sin(2.0 * M_PI * t / pr[2] + pr[3]);
    gval[node[i]] = pr[0] + pr[1] * (sn >= 0.0 ? 1.0 : -1.0);
}

template <typename T>
__global__ void rows_copy_kernel(int n, const long long* __restrict__ idx, const T* __restrict__ src,
                                 T* __restrict__ dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[idx[i]] = src[idx[i]];
}

template <typename T>
__global__ void rows_fill_kernel(int n, const long long* __restrict__ idx, T v, T* __restrict__ dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[idx[i]] = v;
}

__global__ void sub64_kernel(long long n, const double* __restrict__ a, double* __restrict__ b) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] -= a[i];
}

template <typename T>
int rows_copy(ht_ctx* c, T* dst, const T* src) {
    const int n = c->n_dint;
    rows_copy_kernel<T><<<(n + 127) / 128, 128, 0, c->stream>>>(n, c->dint, src, dst); ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    return HT_OK;
}

template <typename T>
int rows_fill(ht_ctx* c, T* dst, T v) {
    const int n = c->n_dint;
    rows_fill_kernel<T><<<(n + 127) / 128, 128, 0, c->stream>>>(n, c->dint, v, dst); ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    return HT_OK;
}

int apply64_raw(ht_ctx* c, int field, double dt, const double* x, double* y, double* dot_part, int* n_part,
                const Scal* sc) {
    HT_TRY(prof_begin(c, field));
    int rc = c->grid.P == 1 ? apply_P<1, double>(c, field, dt, x, y, dot_part, n_part, sc)
                            : apply_P<2, double>(c, field, dt, x, y, dot_part, n_part, sc);
    if (rc != HT_OK) return rc;
    HT_TRY(prof_end(c));
    if (field == HT_TEMP && c->n_well_nodes > 0) return launch_well_apply64(c, dt, x, y, sc);
    return HT_OK;
}

int apply32_raw(ht_ctx* c, int field, float dt, const float* x, float* y, double* dot_part, int* n_part,
                const Scal* sc) {
    HT_TRY(prof_begin(c, field + 2));
    int rc = c->grid.P == 1 ? apply_P<1, float>(c, field, dt, x, y, dot_part, n_part, sc)
                            : apply_P<2, float>(c, field, dt, x, y, dot_part, n_part, sc);
    if (rc != HT_OK) return rc;
    HT_TRY(prof_end(c));
    if (field == HT_TEMP && c->n_well_nodes > 0) return launch_well_apply32(c, dt, x, y, sc);
    return HT_OK;
}

}  // namespace

bool heat_fused_ok(const ht_ctx* c) { return c->n_dint == 0; }

int dint_scatter(ht_ctx* c, double* dst, const double* src) {
    if (c->n_dint == 0) return HT_OK;
    return rows_copy<double>(c, dst, src);
}

int launch_time_dirichlet(ht_ctx* c, double t) {
    for (int f = 0; f < 2; ++f) {
        Grid g = c->grid;
        g.dmask = c->dmask[f];
        for (int face = 0; face < 6; ++face) {
            const ht_ctx::Seasonal& sn = c->seasonal[f][face];
            if (!sn.on) continue;
            const double v = sn.mean + sn.amp * sin(2.0 * M_PI * t / sn.period + sn.phase);
            face_value_kernel<<<64, 256, 0, c->stream>>>(g, face, v, c->g[f]); ++c->n_launch;
            HT_CUDA(c, cudaGetLastError());
        }
    }
    if (c->n_ptemp_nodes > 0) {
        const int n = c->n_ptemp_nodes;
        pile_temp_kernel<<<(n + 127) / 128, 128, 0, c->stream>>>(n, c->ptemp_node, c->ptemp_pile, c->d_ptemp, t,
                                                                 c->g[HT_TEMP]); ++c->n_launch;
        HT_CUDA(c, cudaGetLastError());
    }
    return HT_OK;
}

int launch_apply64(ht_ctx* c, int field, double dt, const double* x, double* y, double* dot_part,
                   int* n_part, const Scal* sc) {
    if (field == HT_TEMP && c->n_dint > 0) {
        if (dot_part) return fail(c, HT_EINVAL, "heat apply with interior Dirichlet rows forms no dot products");
        HT_CUDA(c, cudaMemcpyAsync(c->dint_a64, x, (size_t)c->grid.nn * sizeof(double), cudaMemcpyDeviceToDevice,
                                   c->stream));
        HT_TRY(rows_fill<double>(c, c->dint_a64, 0.0));
        HT_TRY(apply64_raw(c, field, dt, c->dint_a64, y, nullptr, nullptr, sc));
        return rows_copy<double>(c, y, x);
    }
    return apply64_raw(c, field, dt, x, y, dot_part, n_part, sc);
}

int launch_apply32(ht_ctx* c, int field, float dt, const float* x, float* y, double* dot_part,
                   int* n_part, const Scal* sc) {
    if (field == HT_TEMP && c->n_dint > 0) {
        if (dot_part) return fail(c, HT_EINVAL, "heat apply with interior Dirichlet rows forms no dot products");
        HT_CUDA(c, cudaMemcpyAsync(c->dint_a32, x, (size_t)c->grid.nn * sizeof(float), cudaMemcpyDeviceToDevice,
                                   c->stream));
        HT_TRY(rows_fill<float>(c, c->dint_a32, 0.0f));
        HT_TRY(apply32_raw(c, field, dt, c->dint_a32, y, nullptr, nullptr, sc));
        return rows_copy<float>(c, y, x);
    }
    return apply32_raw(c, field, dt, x, y, dot_part, n_part, sc);
}

template <int P, class Op>
static int launch_rhs_two_pass(ht_ctx* c, const Grid& g, const Op& op) {
    // the mass-only cells in float-float (the FP64 rate makes FP64 the slow
    // part here), the Dirichlet cells in FP64, the sum in float-float; the
    // element buffer holds float pairs
    df64* E = reinterpret_cast<df64*>(elem_buffer<double>(c));
    dim3 ci, ng;
    int zi, kl;
    cell_pass_dims(c, g, resident_per_sm<rhs_interior_df_kernel<P>>(), &ci, &zi);
    layer_node_dims(c, g, resident_per_sm<node_emit_df_kernel<P, Op>>(), &ng, &kl);
    const double* scale_c = nullptr;
    double scale_u = 0.0;
    if constexpr (Op::kPlanes) { scale_c = op.cTc; scale_u = op.cT_u; }
    else { scale_u = op.alpha; }
    const float su_hi = (float)scale_u;
    const df64 su(su_hi, (float)(scale_u - (double)su_hi));
    rhs_interior_df_kernel<P><<<ci, dim3(32, 4), 0, c->stream>>>(g, c->edf, op.x, scale_c, su, E, zi); ++c->n_launch;
    if (g.dmask) {
        const long long n_cand = 2LL * ((long long)g.ncy * g.ncz + (long long)g.ncx * g.ncz + (long long)g.ncx * g.ncy);
        rhs_boundary_kernel<P, double, Op, df64><<<(unsigned)((n_cand + 127) / 128), 128, 0, c->stream>>>(g, op, E,
                                                                                                           n_cand);
        ++c->n_launch;
    }
    node_emit_df_kernel<P, Op><<<ng, 128, 0, c->stream>>>(g, E, op, kl); ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    return HT_OK;
}

template <int P>
static int rhs_P(ht_ctx* c, int field, double dt, const double* u_old, double* b) {
    const Grid g = field_grid(c, field);
    const bool two_pass = elem_buffer<double>(c) != nullptr;
    if (field == HT_HEAD) {
        HeadOp<P, double, MODE_RHS> op{};
        op.x = u_old; op.gD = c->g[field]; op.F = c->F[field]; op.y = b;
        op.K = c->K64; op.alpha = c->Ss; op.dt = dt; op.e = c->e64;
        set_geo(op, c);
        if (two_pass) return launch_rhs_two_pass<P>(c, g, op);
        return launch_tile<P, double>(c, g, op, nullptr, nullptr);
    }
    HeatOp<P, double, MODE_RHS> op{};
    op.x = u_old; op.gD = c->g[field]; op.F = c->F[field]; op.y = b;
    op.qs = c->qs64; op.cTc = c->cT64; op.lamc = c->lam64;
    op.cT_u = c->cT_u; op.lam_u = c->lam_u; op.dt = dt; op.cw = c->cw; op.e = c->e64;
    set_geo(op, c);
    if (two_pass) return launch_rhs_two_pass<P>(c, g, op);
    return launch_tile<P, double>(c, g, op, nullptr, nullptr);
}

int launch_rhs(ht_ctx* c, int field, double dt, const double* u_old, double* b) {
    HT_TRY(c->grid.P == 1 ? rhs_P<1>(c, field, dt, u_old, b) : rhs_P<2>(c, field, dt, u_old, b));
    if (field == HT_TEMP && c->n_dint > 0) {
        // lift of the interior rows: b -= A0 g_I on every row (A0 g_I is 0 on
        // the face rows, whose columns it never reaches), then b = g on them
        const size_t nn = (size_t)c->grid.nn;
        HT_CUDA(c, cudaMemsetAsync(c->dint_a64, 0, nn * sizeof(double), c->stream));
        HT_TRY(rows_copy<double>(c, c->dint_a64, c->g[HT_TEMP]));
        HT_TRY(apply64_raw(c, HT_TEMP, dt, c->dint_a64, c->dint_b64, nullptr, nullptr, nullptr));
        sub64_kernel<<<vec_grid(c), kVecThreads, 0, c->stream>>>(c->grid.nn, c->dint_b64, b); ++c->n_launch;
        HT_CUDA(c, cudaGetLastError());
        HT_TRY(rows_copy<double>(c, b, c->g[HT_TEMP]));
    }
    return HT_OK;
}

template <int P>
static int diag_P(ht_ctx* c, int field, double dt, double* D) {
    const Grid g = field_grid(c, field);
    if (field == HT_HEAD) {
        HeadOp<P, double, MODE_DIAG> op{};
        op.y = D; op.K = c->K64; op.alpha = c->Ss; op.dt = dt; op.e = c->e64;
        set_geo(op, c);
        return launch_tile<P, double>(c, g, op, nullptr, nullptr);
    }
    HeatOp<P, double, MODE_DIAG> op{};
    op.y = D; op.qs = c->qs64; op.cTc = c->cT64; op.lamc = c->lam64;
    op.cT_u = c->cT_u; op.lam_u = c->lam_u; op.dt = dt; op.cw = c->cw; op.e = c->e64;
    set_geo(op, c);
    return launch_tile<P, double>(c, g, op, nullptr, nullptr);
}

template <int P>
static int diag32_P(ht_ctx* c, int field, float dt, float* D) {
    const Grid g = field_grid(c, field);
    if (field == HT_HEAD) {
        HeadOp<P, float, MODE_DIAG> op{};
        op.y = D; op.K = c->K32; op.alpha = (float)c->Ss; op.dt = dt; op.e = c->e32;
        set_geo(op, c);
        return launch_tile<P, float>(c, g, op, nullptr, nullptr);
    }
    HeatOp<P, float, MODE_DIAG> op{};
    op.y = D; op.qs = c->qs32; op.cTc = c->cT32; op.lamc = c->lam32;
    op.cT_u = (float)c->cT_u; op.lam_u = (float)c->lam_u; op.dt = dt; op.cw = (float)c->cw; op.e = c->e32;
    set_geo(op, c);
    return launch_tile<P, float>(c, g, op, nullptr, nullptr);
}

int launch_diag32(ht_ctx* c, int field, double dt, float* D) {
    int rc = c->grid.P == 1 ? diag32_P<1>(c, field, (float)dt, D) : diag32_P<2>(c, field, (float)dt, D);
    if (rc != HT_OK) return rc;
    if (field == HT_TEMP && c->n_well_nodes > 0) {
        const int n = c->n_well_nodes;
        well_diag_kernel<float><<<(n + 127) / 128, 128, 0, c->stream>>>(n, c->well_node, c->well_d, dt, D);
        ++c->n_launch;
        HT_CUDA(c, cudaGetLastError());
    }
    if (field == HT_TEMP && c->n_dint > 0) return rows_fill<float>(c, D, 1.0f);
    return HT_OK;
}

// FP64 vector to float pairs, once per residual (the cell kernels read every
// node eight times; the conversion runs on the slow FP64 pipe)
__global__ void split_df_kernel(long long n, const double* __restrict__ a, df64* __restrict__ out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = df_from(a[i]);
}

static int split_df(ht_ctx* c, const double* a, df64** buf) {
    if (!*buf && cudaMalloc(buf, (size_t)c->grid.nn * sizeof(df64)) != cudaSuccess)
        return fail(c, HT_ENOMEM, "float-float operand buffer: allocation failed");
    split_df_kernel<<<vec_grid(c), kVecThreads, 0, c->stream>>>(c->grid.nn, a, *buf); ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    return HT_OK;
}

template <int P, class Op>
static int resid_df_P(ht_ctx* c, const Grid& g, const Op& op, const double* x, const double* b, float* r32,
                      double* part, int* n_part, double dt, const double* wd) {
    df64* E = reinterpret_cast<df64*>(elem_buffer<double>(c));
    dim3 ng;
    int kl;
    layer_node_dims(c, g, resident_per_sm<df_resid_node_kernel<P>>(), &ng, &kl);
    if ((int)(ng.x * ng.y) > c->part_stride) return fail(c, HT_EINVAL, "too many partial sums");
    if constexpr (Op::kPlanes) {
        HT_TRY((launch_heat_planes<P, df64>(c, g, op, LoadSplit{x}, E, nullptr)));
    } else {
        dim3 cg;
        int zl;
        cell_pass_dims(c, g, resident_per_sm<df_cell_kernel<P, Op>>(), &cg, &zl);
        HT_TRY(split_df(c, x, &c->xdf));
        df_cell_kernel<P, Op><<<cg, dim3(32, 4), 0, c->stream>>>(g, op, c->xdf, E, zl); ++c->n_launch;
    }
    df_resid_node_kernel<P><<<ng, 128, 0, c->stream>>>(g, E, x, b, wd, dt, r32, part, c->part_stride, kl);
    ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    *n_part = (int)(ng.x * ng.y);
    return HT_OK;
}

static df64 df_split(double d) {
    const float hi = (float)d;
    return df64(hi, (float)(d - (double)hi));
}

// ---------------------------------------------------------------------------
// Q1 heat operator of one cell in float-float for the outer residual of the
// mixed heat solve (Eq. 4: c_T M + dt lambda K + dt c_w C(q), q = -K_c grad h
// at the 2 x 2 x 2 Gauss points).  Mass and conduction in the element
// eigenbasis of h = [[1, 1], [1, -1]] per axis (the cell matrix is
// (h x h x h)^T diag(c_T MA_l + dt lambda KB_l) (h x h x h)); advection from
// the edge differences of u and of h interpolated to the Gauss points: on a
// Q1 cell the derivative along an axis is the edge difference interpolated
// in the other two directions, and the Gauss weight times N_i sums back the
// same way.  The head gradient is formed from h here, so the stored Gauss
// point velocities are not read.
// ---------------------------------------------------------------------------
struct Q1HeatDf {
    df64 MA[8], KB[8];      // mode eigenvalues: c_T MA_l + (dt lambda) KB_l (KB without dt)
    df64 g0, g1;            // Gauss abscissae on [0, 1]
    df64 fx, fy, fz;        // dt c_w W / H_d^2 (times -K_c per cell)
    df64 cT, dtlam;         // uniform c_T and dt lambda (per-cell arrays when present)
    double dt;
};

__device__ __forceinline__ void gauss2_df(const df64 (&d)[4], df64 g0, df64 g1, df64 (&o)[4]) {
    df64 t[4];
    t[0] = g1 * d[0] + g0 * d[1];   // along i
    t[1] = g0 * d[0] + g1 * d[1];
    t[2] = g1 * d[2] + g0 * d[3];
    t[3] = g0 * d[2] + g1 * d[3];
    o[0] = g1 * t[0] + g0 * t[2];   // along j
    o[1] = g1 * t[1] + g0 * t[3];
    o[2] = g0 * t[0] + g1 * t[2];
    o[3] = g0 * t[1] + g1 * t[3];
}
__device__ __forceinline__ void face_fwd_df(df64 u0, df64 u1, df64 u2, df64 u3, df64 (&F)[4]) {
    const df64 s0 = u0 + u1, d0 = u0 - u1, s1 = u2 + u3, d1 = u2 - u3;
    F[0] = s0 + s1;
    F[1] = d0 + d1;
    F[2] = s0 - s1;
    F[3] = d0 - d1;
}
__device__ __forceinline__ void face_bwd_df(const df64 (&G)[4], df64 (&u)[4]) {
    const df64 t0 = G[0] + G[2], t1 = G[1] + G[3], w0 = G[0] - G[2], w1 = G[1] - G[3];
    u[0] = t0 + t1;
    u[1] = t0 - t1;
    u[2] = w0 + w1;
    u[3] = w0 - w1;
}

__global__ void __launch_bounds__(128) q1_heat_df_cell_kernel(const Grid g, const df64* __restrict__ x,
                                                              const df64* __restrict__ h,
                                                              const double* __restrict__ K,
                                                              const double* __restrict__ cTc,
                                                              const double* __restrict__ lamc, const Q1HeatDf k,
                                                              df64* __restrict__ E) {
    const long long nc = g.nc;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < nc;
         c += (long long)gridDim.x * blockDim.x) {
        const int cx = (int)(c % g.ncx), cy = (int)((c / g.ncx) % g.ncy), cz = (int)(c / ((long long)g.ncx * g.ncy));
        const long long base = cx + (long long)g.Nx * (cy + (long long)g.Ny * cz);
        const long long NX = g.Nx, NXY = (long long)g.Nx * g.Ny;
        const bool chk = g.dmask != 0 && (cx == 0 || cx == g.ncx - 1 || cy == 0 || cy == g.ncy - 1 || cz == 0 ||
                                          cz == g.ncz - 1);
        df64 U[2][4], H[2][4];   // [plane c][corner a + 2 b]
#pragma unroll
        for (int pc = 0; pc < 2; ++pc)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int a = q & 1, b = q >> 1;
                const long long id = base + a + NX * b + NXY * pc;
                df64 uv = ldg_any<df64>(x + id);
                if (chk && on_dir(g, cx + a, cy + b, cz + pc)) uv = df64(0);
                U[pc][q] = uv;
                H[pc][q] = ldg_any<df64>(h + id);
            }
        // mass + conduction in the eigenbasis
        const df64 cT = cTc ? df_from(ldro(cTc + c)) : k.cT;
        const df64 dtlam = lamc ? df_from(k.dt * ldro(lamc + c)) : k.dtlam;
        df64 F0[4], F1[4], bot[4], top[4];
        face_fwd_df(U[0][0], U[0][1], U[0][2], U[0][3], F0);
        face_fwd_df(U[1][0], U[1][1], U[1][2], U[1][3], F1);
        {
            df64 bh[4], th[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const df64 lo = (F0[q] + F1[q]) * (cT * k.MA[q] + dtlam * k.KB[q]);
                const df64 hi = (F0[q] - F1[q]) * (cT * k.MA[q + 4] + dtlam * k.KB[q + 4]);
                bh[q] = lo + hi;
                th[q] = lo - hi;
            }
            face_bwd_df(bh, bot);
            face_bwd_df(th, top);
        }
        // advection: edge differences of u and h (corner index a + 2 b, plane c)
        df64 du[4], dh[4], iu[4], ih[4], pr[4], rx[4], ry[4], rz[4];
        du[0] = U[0][1] - U[0][0]; du[1] = U[0][3] - U[0][2]; du[2] = U[1][1] - U[1][0]; du[3] = U[1][3] - U[1][2];
        dh[0] = H[0][1] - H[0][0]; dh[1] = H[0][3] - H[0][2]; dh[2] = H[1][1] - H[1][0]; dh[3] = H[1][3] - H[1][2];
        gauss2_df(du, k.g0, k.g1, iu);
        gauss2_df(dh, k.g0, k.g1, ih);
#pragma unroll
        for (int q = 0; q < 4; ++q) pr[q] = iu[q] * ih[q];
        gauss2_df(pr, k.g0, k.g1, rx);
        du[0] = U[0][2] - U[0][0]; du[1] = U[0][3] - U[0][1]; du[2] = U[1][2] - U[1][0]; du[3] = U[1][3] - U[1][1];
        dh[0] = H[0][2] - H[0][0]; dh[1] = H[0][3] - H[0][1]; dh[2] = H[1][2] - H[1][0]; dh[3] = H[1][3] - H[1][1];
        gauss2_df(du, k.g0, k.g1, iu);
        gauss2_df(dh, k.g0, k.g1, ih);
#pragma unroll
        for (int q = 0; q < 4; ++q) pr[q] = iu[q] * ih[q];
        gauss2_df(pr, k.g0, k.g1, ry);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            du[q] = U[1][q] - U[0][q];
            dh[q] = H[1][q] - H[0][q];
        }
        gauss2_df(du, k.g0, k.g1, iu);
        gauss2_df(dh, k.g0, k.g1, ih);
#pragma unroll
        for (int q = 0; q < 4; ++q) pr[q] = iu[q] * ih[q];
        gauss2_df(pr, k.g0, k.g1, rz);
        const df64 mk = -df_from(ldro(K + c));
        const df64 fx = mk * k.fx, fy = mk * k.fy, fz = mk * k.fz;
        const int ncl = (int)nc;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int a = q & 1, bb = q >> 1;
            const df64 zq = fz * rz[q];
            const df64 b0 = bot[q] + (fx * rx[bb] + (fy * ry[a] + zq));
            const df64 t0 = top[q] + (fx * rx[bb + 2] + (fy * ry[a + 2] + zq));
            E[(size_t)q * ncl + c] = b0;
            E[(size_t)(q + 4) * ncl + c] = t0;
        }
    }
}

static Q1HeatDf q1_heat_df_const(const ht_ctx* c, double dt) {
    Q1HeatDf k{};
    const double* H = c->H;
    double m1[3][2], k1[3][2];
    for (int d = 0; d < 3; ++d) {
        m1[d][0] = H[d];
        m1[d][1] = H[d] / 3.0;
        k1[d][0] = 0.0;
        k1[d][1] = 4.0 / H[d];
    }
    auto split = [](double v) {
        const float hi = (float)v;
        return df64(hi, (float)(v - (double)hi));
    };
    for (int cz = 0; cz < 2; ++cz)
        for (int by = 0; by < 2; ++by)
            for (int ax = 0; ax < 2; ++ax) {
                const int l = ax + 2 * by + 4 * cz;
                const double M = m1[0][ax] * m1[1][by] * m1[2][cz];
                const double Kl = k1[0][ax] * m1[1][by] * m1[2][cz] + m1[0][ax] * k1[1][by] * m1[2][cz] +
                                  m1[0][ax] * m1[1][by] * k1[2][cz];
                k.MA[l] = split(M / 64.0);
                k.KB[l] = split(Kl / 64.0);
            }
    const double d = 0.5 / sqrt(3.0);
    k.g0 = split(0.5 - d);
    k.g1 = split(0.5 + d);
    const double W = H[0] * H[1] * H[2] / 8.0;
    k.fx = split(dt * c->cw * W / (H[0] * H[0]));
    k.fy = split(dt * c->cw * W / (H[1] * H[1]));
    k.fz = split(dt * c->cw * W / (H[2] * H[2]));
    k.cT = split(c->cT_u);
    k.dtlam = split(dt * c->lam_u);
    k.dt = dt;
    return k;
}

template <int P>
static int resid_df_field(ht_ctx* c, int field, double dt, const double* x, const double* b, float* r32,
                          double* part, int* n_part) {
    const Grid g = field_grid(c, field);
    if (P == 1 && field == HT_TEMP && !c->graded) {
        // Q1 heat: the cell kernel above, then the node gather of the
        // residual (wells and Dirichlet rows there)
        df64* E = reinterpret_cast<df64*>(elem_buffer<double>(c));
        dim3 ng;
        int kl;
        layer_node_dims(c, g, resident_per_sm<df_resid_node_kernel<P>>(), &ng, &kl);
        if ((int)(ng.x * ng.y) > c->part_stride) return fail(c, HT_EINVAL, "too many partial sums");
        long long blocks = (g.nc + 127) / 128;
        const long long cap = (long long)(c->num_sms > 0 ? c->num_sms : 148) * 16;
        if (blocks > cap) blocks = cap;
        HT_TRY(split_df(c, x, &c->xdf));
        HT_TRY(split_df(c, c->h, &c->hdf));
        q1_heat_df_cell_kernel<<<(unsigned)blocks, 128, 0, c->stream>>>(g, c->xdf, c->hdf, c->K64, c->cT64,
                                                                         c->lam64, q1_heat_df_const(c, dt), E);
        ++c->n_launch;
        df_resid_node_kernel<P><<<ng, 128, 0, c->stream>>>(g, E, x, b, c->wdn64, dt, r32, part, c->part_stride, kl);
        ++c->n_launch;
        HT_CUDA(c, cudaGetLastError());
        *n_part = (int)(ng.x * ng.y);
        return HT_OK;
    }
    if (field == HT_HEAD) {
        HeadOp<P, df64, MODE_APPLY, double> op{};
        op.K = c->K64; op.alpha = df_split(c->Ss); op.dt = df_split(dt); op.e = c->edf;
        set_geo(op, c);
        return resid_df_P<P>(c, g, op, x, b, r32, part, n_part, dt, nullptr);
    }
    HeatOp<P, df64, MODE_APPLY, double> op{};
    op.qs = c->qs64; op.cTc = c->cT64; op.lamc = c->lam64;
    op.cT_u = df_split(c->cT_u); op.lam_u = df_split(c->lam_u); op.dt = df_split(dt); op.cw = df_split(c->cw);
    op.e = c->edf;
    set_geo(op, c);
    op.g_nc = g.nc;
    return resid_df_P<P>(c, g, op, x, b, r32, part, n_part, dt, c->wdn64);
}

int launch_resid_df(ht_ctx* c, int field, double dt, const double* x, const double* b, float* r32,
                    double* part, int* n_part) {
    if (!c->E64) return fail(c, HT_EINVAL, "no element buffer");
    return c->grid.P == 1 ? resid_df_field<1>(c, field, dt, x, b, r32, part, n_part)
                          : resid_df_field<2>(c, field, dt, x, b, r32, part, n_part);
}

int launch_diag(ht_ctx* c, int field, double dt, double* D) {
    int rc = c->grid.P == 1 ? diag_P<1>(c, field, dt, D) : diag_P<2>(c, field, dt, D);
    if (rc != HT_OK) return rc;
    if (field == HT_TEMP && c->n_well_nodes > 0) HT_TRY(launch_well_diag(c, dt, D));
    if (field == HT_TEMP && c->n_dint > 0) return rows_fill<double>(c, D, 1.0);
    return HT_OK;
}

// Q1: the derivative along an axis is the same at both Gauss points of that
// axis, the edge difference (u1 - u0) / H interpolated in the other two
// directions, so the 24 values of a cell come from 12 edge differences and
// three bilinear interpolations
__global__ void __launch_bounds__(128) darcy_qp_q1_kernel(const Grid g, const double* __restrict__ h,
                                                          const double* __restrict__ K, const Elem<double> e,
                                                          double* __restrict__ qs64, float* __restrict__ qs32) {
    constexpr int NQ = 8;
    const double B[2][2] = {{e.B[0][0], e.B[0][1]}, {e.B[1][0], e.B[1][1]}};
    // out[i][j] = sum_a sum_b B[i][a] B[j][b] d[a][b]
    auto interp = [&](const double (&d)[2][2], double (&out)[2][2]) {
        double t[2][2];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int j = 0; j < 2; ++j) t[a][j] = fma(B[j][1], d[a][1], B[j][0] * d[a][0]);
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) out[i][j] = fma(B[i][1], t[1][j], B[i][0] * t[0][j]);
    };
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < g.nc;
         c += (long long)gridDim.x * blockDim.x) {
        const int cx = (int)(c % g.ncx), cy = (int)((c / g.ncx) % g.ncy), cz = (int)(c / ((long long)g.ncx * g.ncy));
        double u[8];
        gather<1, double>(g, h, cx, cy, cz, false, u);   // u[a + 2 (b + 2 c)]
        const double Kc = K[c];
        double dx[2][2], dy[2][2], dz[2][2];   // dx[b][c], dy[a][c], dz[a][b]
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                dx[i][j] = u[1 + 2 * (i + 2 * j)] - u[0 + 2 * (i + 2 * j)];
                dy[i][j] = u[i + 2 * (1 + 2 * j)] - u[i + 2 * (0 + 2 * j)];
                dz[i][j] = u[i + 2 * (j + 2)] - u[i + 2 * j];
            }
        double gx[2][2], gy[2][2], gz[2][2];   // gx[qy][qz], gy[qx][qz], gz[qx][qy]
        interp(dx, gx);
        interp(dy, gy);
        interp(dz, gz);
        double ih[3] = {e.invH[0], e.invH[1], e.invH[2]};
        if (g.geo64)
            for (int d = 0; d < 3; ++d) ih[d] = g.geo64[(d + 1) * g.nc + c];
        const double sx = -Kc * ih[0], sy = -Kc * ih[1], sz = -Kc * ih[2];
#pragma unroll
        for (int qz = 0; qz < 2; ++qz)
#pragma unroll
            for (int qy = 0; qy < 2; ++qy)
#pragma unroll
                for (int qx = 0; qx < 2; ++qx) {
                    const int qi = qx + 2 * (qy + 2 * qz);
                    const double q0 = sx * gx[qy][qz], q1 = sy * gy[qx][qz], q2 = sz * gz[qx][qy];
                    qs64[(0 * NQ + qi) * g.nc + c] = q0;
                    qs64[(1 * NQ + qi) * g.nc + c] = q1;
                    qs64[(2 * NQ + qi) * g.nc + c] = q2;
                    qs32[(0 * NQ + qi) * g.nc + c] = (float)q0;
                    qs32[(1 * NQ + qi) * g.nc + c] = (float)q1;
                    qs32[(2 * NQ + qi) * g.nc + c] = (float)q2;
                }
    }
}

int launch_darcy_qp(ht_ctx* c, const double* h) {
    const Grid g = field_grid(c, HT_HEAD);
    const int threads = 128;
    long long blocks = (g.nc + threads - 1) / threads;
    const long long cap = (long long)c->num_sms * 16;
    if (blocks > cap) blocks = cap;
    if (c->grid.P == 1)
        darcy_qp_q1_kernel<<<(int)blocks, threads, 0, c->stream>>>(g, h, c->K64, c->e64, c->qs64, c->qs32);
    else
        darcy_qp_kernel<2><<<(int)blocks, threads, 0, c->stream>>>(g, h, c->K64, c->e64, c->qs64, c->qs32);
    ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    return HT_OK;
}

int launch_cell_flux(ht_ctx* c, const double* h, int comp, double* out) {
    const Grid g = field_grid(c, HT_HEAD);
    CentreBasis cb{};
    if (c->grid.P == 1) {
        cb.v[0] = 0.5; cb.v[1] = 0.5; cb.d[0] = -1.0; cb.d[1] = 1.0;
    } else {
        // Q2 basis on nodes {0, 1/2, 1} evaluated at the cell centre
        cb.v[0] = 0.0; cb.v[1] = 1.0; cb.v[2] = 0.0;
        cb.d[0] = -1.0; cb.d[1] = 0.0; cb.d[2] = 1.0;
    }
    const int threads = 256;
    long long blocks = (g.nc + threads - 1) / threads;
    const long long cap = (long long)c->num_sms * 16;
    if (blocks > cap) blocks = cap;
    const double invH = 1.0 / c->H[comp];
    if (c->grid.P == 1)
        cell_flux_kernel<1><<<(int)blocks, threads, 0, c->stream>>>(g, h, c->K64, cb, invH, comp, out);
    else
        cell_flux_kernel<2><<<(int)blocks, threads, 0, c->stream>>>(g, h, c->K64, cb, invH, comp, out);
    ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    return HT_OK;
}

int launch_well_apply64(ht_ctx* c, double dt, const double* x, double* y, const Scal* sc) {
    const int n = c->n_well_nodes;
    well_apply_kernel<double><<<(n + 127) / 128, 128, 0, c->stream>>>(n, c->well_node, c->well_d, dt, x, y, sc); ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    return HT_OK;
}

int launch_well_apply32(ht_ctx* c, float dt, const float* x, float* y, const Scal* sc) {
    const int n = c->n_well_nodes;
    well_apply_kernel<float><<<(n + 127) / 128, 128, 0, c->stream>>>(n, c->well_node, c->well_d, dt, x, y, sc); ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    return HT_OK;
}

int launch_well_diag(ht_ctx* c, double dt, double* D) {
    const int n = c->n_well_nodes;
    well_diag_kernel<double><<<(n + 127) / 128, 128, 0, c->stream>>>(n, c->well_node, c->well_d, dt, D); ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    return HT_OK;
}

int launch_loads(ht_ctx* c, double t) {
    const long long nn = c->grid.nn;
    const int grid = vec_grid(c);
    for (int f = 0; f < 2; ++f) {
        add_kernel<<<grid, kVecThreads, 0, c->stream>>>(nn, c->Fstat[f], c->extra[f], c->F[f]); ++c->n_launch;
        HT_CUDA(c, cudaGetLastError());
    }
    if (c->n_pile_nodes > 0) {
        // pile nodes: F_T = Fstat + extra + sum_s q_l,s(t) w_s (unique nodes)
        const int n = c->n_pile_nodes;
        pile_load_kernel<<<(n + 127) / 128, 128, 0, c->stream>>>(n, c->pile_node, c->pile_off, c->pile_src,
                                                                 c->pile_w, c->d_piles, t, c->F[HT_TEMP],
                                                                 c->F[HT_TEMP]); ++c->n_launch;
        HT_CUDA(c, cudaGetLastError());
    }
    return launch_time_dirichlet(c, t);
}

// ---------------------------------------------------------------------------
// Allocation-free head apply with x^T A x (ht_head_apply_dot_noalloc).
//
// Scratch for the per-tile partial sums of x^T A x lives in this fixed,
// file-scope device array instead of memory from cudaMalloc.  Every GPU that
// loads the library holds it until the process exits.  Host code cannot use
// the symbol itself as a device address: its device address is looked up
// once per device with cudaGetSymbolAddress, with that device current.
// ---------------------------------------------------------------------------
static __device__ __align__(256) double ht_noalloc_part[kNoAllocMaxTiles];

namespace {
std::mutex g_noalloc_mu;
double* g_noalloc_addr[kNoAllocMaxDevices] = {nullptr};

__global__ void noalloc_reduce_kernel(const double* __restrict__ part, int n, double* __restrict__ out) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
    s = block_sum(s);
    if (threadIdx.x == 0) *out = s;
}

template <int P>
int noalloc_P(const Grid& g, const Elem<double>& e, double Ss, double dt, const double* K, const double* x,
              double* y, double* xAx, double* part, int num_sms, cudaStream_t stream, char* msg, size_t msg_len) {
    using Sh = TileShape<P, kCXM, kCYM>;
    const int tx = (g.Nx + Sh::TX - 1) / Sh::TX, ty = (g.Ny + Sh::TY - 1) / Sh::TY;
    const int target = 2 * (num_sms > 0 ? num_sms : 148);
    int chunks = (target + tx * ty - 1) / (tx * ty);
    chunks = chunks < 1 ? 1 : (chunks > g.ncz ? g.ncz : chunks);
    const int zc = (g.ncz + chunks - 1) / chunks;
    chunks = (g.ncz + zc - 1) / zc;
    const long long tiles = (long long)tx * ty * chunks;
    if (tiles > kNoAllocMaxTiles) {
        if (msg && msg_len) snprintf(msg, msg_len, "mesh needs %lld tiles; the static scratch holds %d", tiles,
                                     kNoAllocMaxTiles);
        return HT_EINVAL;
    }
    HeadOp<P, double, MODE_APPLY> op{};
    op.x = x; op.y = y; op.K = K; op.alpha = Ss; op.dt = dt; op.e = e;
    constexpr int n = P + 1, NL = n * n * n;
    const size_t smem = (size_t)kCXM * kCYM * NL * sizeof(double);
    auto kern = tile_kernel<P, double, kCXM, kCYM, HeadOp<P, double, MODE_APPLY>>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err == cudaSuccess) {
        kern<<<dim3(tx, ty, chunks), kCXM * kCYM, smem, stream>>>(g, op, zc, part, nullptr);
        err = cudaGetLastError();
    }
    if (err == cudaSuccess) {
        noalloc_reduce_kernel<<<1, 256, 0, stream>>>(part, (int)tiles, xAx);
        err = cudaGetLastError();
    }
    if (err != cudaSuccess) {
        if (msg && msg_len) snprintf(msg, msg_len, "CUDA error: %s", cudaGetErrorString(err));
        return HT_ECUDA;
    }
    return HT_OK;
}
}  // namespace

int noalloc_head_apply_dot(const Grid& g, const Elem<double>& e, double Ss, double dt, const double* K,
                           const double* x, double* y, double* xAx, int device, cudaStream_t stream, char* msg,
                           size_t msg_len) {
    if (device < 0 || device >= kNoAllocMaxDevices) {
        if (msg && msg_len) snprintf(msg, msg_len, "device %d out of range", device);
        return HT_EINVAL;
    }
    // the caller's current device is restored on every return path
    struct DeviceRestore {
        int prev = -1;
        ~DeviceRestore() { if (prev >= 0) cudaSetDevice(prev); }
    } restore;
    cudaError_t err = cudaGetDevice(&restore.prev);
    if (err != cudaSuccess) restore.prev = -1;
    else if (restore.prev != device) err = cudaSetDevice(device);
    else restore.prev = -1;        // already current: nothing to restore
    double* part = nullptr;
    int num_sms = 0;
    if (err == cudaSuccess) {
        // one-time set-up per device: the device address of the static scratch
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_addr[device]) {
            void* addr = nullptr;
            err = cudaGetSymbolAddress(&addr, ht_noalloc_part);
            if (err == cudaSuccess) g_noalloc_addr[device] = static_cast<double*>(addr);
        }
        part = g_noalloc_addr[device];
    }
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device);
    if (err != cudaSuccess) {
        if (msg && msg_len) snprintf(msg, msg_len, "CUDA error: %s", cudaGetErrorString(err));
        return HT_ECUDA;
    }
    return g.P == 1 ? noalloc_P<1>(g, e, Ss, dt, K, x, y, xAx, part, num_sms, stream, msg, msg_len)
                    : noalloc_P<2>(g, e, Ss, dt, K, x, y, xAx, part, num_sms, stream, msg, msg_len);
}

}  // namespace ht
