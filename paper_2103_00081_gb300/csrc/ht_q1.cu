// Single-pass Jacobi-preconditioned conjugate gradient iteration of the Q1
// head system (S_s M + dt K_K) d = r of the FP32 inner solves (Eq. 3 in head
// form), one launch per iteration.
//
// Method.  The iteration is the single-reduction form of preconditioned CG
// (Chronopoulos and Gear, 1989): with u = D^-1 r,
//     p_i = u_i + beta_i p_{i-1},   s_i = A p_i,
//     x_{i+1} = x_i + alpha_i p_i,  r_{i+1} = r_i - alpha_i s_i,
//     gamma_{i+1} = r_{i+1} . u_{i+1},   delta_{i+1} = u_{i+1}^T A u_{i+1},
//     beta_{i+1} = gamma_{i+1} / gamma_i,
//     alpha_{i+1} = gamma_{i+1} / (delta_{i+1} - beta_{i+1} gamma_{i+1} / alpha_i).
// It produces the iterates of classical PCG (the two scalars are the same
// quantities rewritten), but its two inner products are taken together, so
// an iteration needs one global reduction instead of two and fits in one
// kernel.  Nothing but x, r and p is stored (r and p in two copies: a CTA
// reads them on a halo that neighbouring CTAs own, so an iteration reads
// one copy and writes the other): D is formed from the cell
// conductivities on the fly, s = A p is recomputed on a tile plus a halo,
// and delta is the sum of the element energies u_e^T A_e u_e (in the
// element eigenbasis below), which needs no assembled A u.  Per node and
// iteration the kernel reads x, r, p and the cell K (about one cell per
// node) and writes x, r, p: 28 bytes in FP32.
//
// Element operator.  On a uniform axis-aligned Q1 cell the 1D mass and
// stiffness matrices m = H/6 [[2,1],[1,2]] and k = 1/H [[1,-1],[-1,1]] are
// both diagonalised by h = [[1,1],[1,-1]]: h m h^T = diag(H, H/3) and
// h k h^T = diag(0, 4/H), with h^-1 = h^T / 2.  So the cell matrix
// alpha M_e + beta_c K_e of the tensor-product element is
//     (h x h x h)^T diag(lambda_l) (h x h x h),
//     lambda_l = (alpha M_l + beta_c K_l) / 64,
// with M_l = mx_a my_b mz_c and K_l = kx_a my_b mz_c + mx_a ky_b mz_c +
// mx_a my_b kz_c for the mode l = (a, b, c) -- additions and subtractions
// only, plus one scaling per mode.
//
// Tiling.  A CTA owns a tile of at most 28 x 20 node columns and a chunk of
// node planes, and marches upward through it.  Per plane step it forms
// p on the tile plus one node on the low side and two on the high side,
// transforms each cell face in x and y once (shared by the cells above and
// below), combines two faces into a cell in z, and gathers the four face
// contributions of every node.  Loads of the next planes are in flight
// (cp.async) while a plane is computed.  Every owned value is produced by
// one thread in a fixed order, and the per-CTA partial sums are reduced by
// the last CTA in a fixed order, so the iteration is deterministic.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <type_traits>

#include "ht_device.cuh"
#include "ht_internal.cuh"

namespace ht {
namespace {

constexpr int kBX = 32, kBY = 8;    // threads of the heat kernel: lanes along x, warps along y
constexpr int kRows = 3;            // rows of a thread of the heat kernel
constexpr int kSX = 32, kSY = 24;   // shared plane: kRows * kBY rows of 32

struct Q1HeadConst {
    float A[8], B[8];   // lambda_l = A_l + (dt K_c) B_l, mode l = a + 2 b + 4 c
    float am3;          // alpha * diag(M_e)
    float dk3;          // dt * diag(K_e)
    float2 A2[8], B2[8];   // the same, each value twice (operands of the packed FP32 form)
};


// grid-barrier state of the persistent batched CG (zeroed before each launch)
struct Q1BatchSync {
    unsigned count;     // arrivals at the running barrier
    unsigned gen;       // barrier generation
    int active[2];      // problems still running, by iteration parity
    int running;        // problems still running when the launch ended
    int err;            // 1: a barrier wait ran out of its budget
    int err_cta;        // the CTA whose wait ran out first
    int pad;
};

// one problem of the persistent batched CG
struct Q1BatchProb {
    Grid g;                      // dmask of the head field
    const float* K;
    float* x;
    float* r[2];                 // the two copies of r and p (iteration parity)
    float* p[2];
    Q1HeadConst cst;
    int ntx, nty, nzc, item0, nitems;
    double* part;                // partial sums [3][stride]
    int stride;
    Scal* s;
};

__device__ __forceinline__ void cp_async4(float* sdst, const float* gsrc, bool valid) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    const int n = valid ? 4 : 0;   // 0: no bytes are read, the word is zero-filled
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gsrc), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

// h x h on the four corners u(a, b), corner index a + 2 b
__device__ __forceinline__ void face_fwd(float u0, float u1, float u2, float u3, float (&F)[4]) {
    const float s0 = u0 + u1, d0 = u0 - u1, s1 = u2 + u3, d1 = u2 - u3;
    F[0] = s0 + s1;
    F[1] = d0 + d1;
    F[2] = s0 - s1;
    F[3] = d0 - d1;
}
// (h x h)^T back to the corners
__device__ __forceinline__ void face_bwd(const float (&G)[4], float (&u)[4]) {
    const float t0 = G[0] + G[2], t1 = G[1] + G[3], w0 = G[0] - G[2], w1 = G[1] - G[3];
    u[0] = t0 + t1;
    u[1] = t0 - t1;
    u[2] = w0 + w1;
    u[3] = w0 - w1;
}

__device__ __forceinline__ int cells_along(int i, int N) { return (i > 0) + (i < N - 1); }

// Flags of one (row, lane) slot of a tile, fixed for the whole march.
enum : unsigned {
    F_OWN = 1u,        // owned node (and owned face)
    F_R1 = 2u,         // node of the s / u region
    F_NIN = 4u,        // node inside the mesh (x, y)
    F_FIN = 8u,        // face (cell column) inside the mesh
    F_KIN = 16u,       // cell of the K slot inside the mesh
    F_DXY = 32u,       // node on a Dirichlet face of x or y
};

// ---------------------------------------------------------------------------
// CG tile: two consecutive node rows per thread, 16 warps, 32 x 32 slots
// (owned tiles of up to 29 x 29 node columns).  A thread's rows R = 2 ty and
// 2 ty + 1 are processed together in packed FP32 (the x and y halves of
// each float2); the row above the pair and the row below it belong to the
// neighbouring warps and cross through small per-warp rows in shared
// memory; horizontal neighbours move by warp shuffles.
// ---------------------------------------------------------------------------
constexpr int kCgBY = 16;                       // warps (two rows each)
constexpr int kCgThreads = 32 * kCgBY;
constexpr int k4SX = 32, k4SY = 2 * kCgBY, k4St = 6;
constexpr int k4TX = k4SX - 3, k4TY = k4SY - 3;   // largest owned tile (node columns)
constexpr int k4BY = kCgBY;

struct Q1Smem4 {
    float ld_r[k4St][k4SY][k4SX];
    float ld_p[k4St][k4SY][k4SX];
    float ld_x[k4St][k4SY][k4SX];
    float ld_k[k4St][k4SY][k4SX];
    float pc0[k4BY][k4SX];   // p at the plane of stage A, first row of each warp
    float us0[k4BY][k4SX];   // u at the plane of stage B, first row of each warp
    float sc2[k4BY][k4SX];   // corner-2 / corner-3 contributions of each warp's last row
    float sc3[k4BY][k4SX];
};

__device__ __forceinline__ void cp_async_wait_ring4() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(k4St - 1) : "memory");
}

__device__ __forceinline__ float rcp_approx(float v) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

// Packed FP32 helpers (two values per instruction: the x component is row
// 2 ty, the y component row 2 ty + 1).  Masks multiply instead of selecting,
// and the per-step energy of a row pair is added to delta once per plane.
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b with one rounding
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }

__device__ __forceinline__ void face_fwd2(float2 u0, float2 u1, float2 u2, float2 u3, float2 (&F)[4]) {
    const float2 s0 = add2(u0, u1), d0 = sub2(u0, u1), s1 = add2(u2, u3), d1 = sub2(u2, u3);
    F[0] = add2(s0, s1);
    F[1] = add2(d0, d1);
    F[2] = sub2(s0, s1);
    F[3] = sub2(d0, d1);
}
__device__ __forceinline__ void face_bwd2(const float2 (&G)[4], float2 (&u)[4]) {
    const float2 t0 = add2(G[0], G[2]), t1 = add2(G[1], G[3]), w0 = sub2(G[0], G[2]), w1 = sub2(G[1], G[3]);
    u[0] = add2(t0, t1);
    u[1] = sub2(t0, t1);
    u[2] = add2(w0, w1);
    u[3] = sub2(w0, w1);
}
__device__ __forceinline__ float2 shfl_down2(float2 v) {
    return f2(__shfl_down_sync(0xffffffffu, v.x, 1), __shfl_down_sync(0xffffffffu, v.y, 1));
}
__device__ __forceinline__ void cp_async4n(float* sdst, const float* gsrc, int nbytes) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gsrc), "r"(nbytes) : "memory");
}

// One CTA's share of a CG iteration: node planes [k0, k1) of the owned tile
// (bx, by) of node columns, marched upward; adds the share's gamma, delta and
// rho to the thread's accumulators.
template <bool FIRST>
__device__ __forceinline__ void q1_cg_tile2p(const Grid& g, const float* __restrict__ K, float* __restrict__ x,
                                             const float* __restrict__ r, const float* __restrict__ p,
                                             float* __restrict__ r_out, float* __restrict__ p_out,
                                             const Q1HeadConst& cst, const int bx, const int by, const int ntx,
                                             const int nty, const int k0, const int k1, const float alpha,
                                             const float beta, Q1Smem4& sm, float2& gam, float2& del,
                                             float2& rho) {
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i0 = (int)((long long)bx * g.Nx / ntx), i1 = (int)((long long)(bx + 1) * g.Nx / ntx);
    const int j0 = (int)((long long)by * g.Ny / nty), j1 = (int)((long long)(by + 1) * g.Ny / nty);
    const int w = i1 - i0, h = j1 - j0;
    __syncthreads();   // the previous share is done with the shared planes
    const int NXY = g.Nx * g.Ny, CXY = g.ncx * g.ncy;
    const int dm = g.dmask;
    const int mbeg = k0 - 2, mend = k1 + 1;
    const int R0 = 2 * ty;
    const int tyn = ty + 1 < k4BY ? ty + 1 : ty;
    const int typ = ty > 0 ? ty - 1 : 0;
    const int Rext = R0 + 2 < k4SY ? R0 + 2 : k4SY - 1;

    // per row: node and cell offsets in a plane (0 where outside: the copy
    // size is then 0), load sizes and masks
    int nofs[2], kofs[2], nsz[2], xsz[2], ksz[2];
    bool own[2];
    float lmv[2], amv[2], omv[2], fmv[2], emv[2];
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        const int R = R0 + b, C = tx;
        const int gi = i0 + C - 1, gj = j0 + R - 1;
        const bool o = R >= 1 && R <= h && C >= 1 && C <= w;
        const bool nin = gi >= 0 && gi < g.Nx && gj >= 0 && gj < g.Ny;
        const bool fin = gi >= 0 && gi < g.ncx && gj >= 0 && gj < g.ncy;
        const bool kin = gi - 1 >= 0 && gi - 1 < g.ncx && gj - 1 >= 0 && gj - 1 < g.ncy;
        const bool dxy = ((dm & 1) && gi == 0) || ((dm & 2) && gi == g.Nx - 1) || ((dm & 4) && gj == 0) ||
                         ((dm & 8) && gj == g.Ny - 1);
        own[b] = o;
        nofs[b] = nin ? gi + g.Nx * gj : 0;
        kofs[b] = kin ? (gi - 1) + g.ncx * (gj - 1) : 0;
        nsz[b] = nin ? 4 : 0;
        xsz[b] = nin && o ? 4 : 0;
        ksz[b] = kin ? 4 : 0;
        lmv[b] = nin && !dxy ? 1.0f : 0.0f;
        amv[b] = nin ? cst.am3 * (float)(cells_along(gi, g.Nx) * cells_along(gj, g.Ny)) : 1.0f;
        omv[b] = o ? 1.0f : 0.0f;
        fmv[b] = fin ? 1.0f : 0.0f;
        emv[b] = o && fin ? 1.0f : 0.0f;
    }
    const float2 lm = f2(lmv[0], lmv[1]), amn = f2(amv[0], amv[1]), om = f2(omv[0], omv[1]);
    const float2 fm = f2(fmv[0], fmv[1]), em = f2(emv[0], emv[1]);
    const float2 alpha2 = f2(alpha, alpha), beta2 = f2(beta, beta), nalpha2 = f2(-alpha, -alpha);
    const float2 dk2 = f2(cst.dk3, cst.dk3);

    auto issue = [&](int q, int st) {
        if (q <= mend) {
            const bool plane_ok = q >= 0 && q < g.Nz;
            const bool layer_ok = q >= 0 && q < g.ncz;
            const int pofs = plane_ok ? NXY * q : 0, cofs = layer_ok ? CXY * q : 0;
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const int R = R0 + b;
                const int id = nofs[b] + pofs, kid = kofs[b] + cofs;
                const int n1 = plane_ok ? nsz[b] : 0;
                cp_async4n(&sm.ld_r[st][R][tx], r + id, n1);
                if (!FIRST) cp_async4n(&sm.ld_p[st][R][tx], p + id, n1);
                cp_async4n(&sm.ld_x[st][R][tx], x + id, plane_ok ? xsz[b] : 0);
                cp_async4n(&sm.ld_k[st][R][tx], K + kid, layer_ok ? ksz[b] : 0);
            }
        }
        cp_async_commit();
    };

    const float2 z2 = f2(0.0f, 0.0f);
    float2 S_prev = z2, hr = z2, hp = z2, hdi = z2, hm = z2, hx = z2, us = z2;
    float2 Fp[4], Tp[4], Gp[4];
    float2 Kf1 = z2, Kf2 = z2, Kf3 = z2;
#pragma unroll
    for (int q = 0; q < 4; ++q) Fp[q] = Tp[q] = Gp[q] = z2;

    // energies of cell layer lc of the owned faces: u at planes lc (its
    // transforms in Gp) and lc + 1 (us, the row above from us0)
    auto energies = [&](bool add, float2 Kl) {
        const float ue = sm.us0[tyn][tx];
        const float2 ur = shfl_down2(us);
        const float uer = __shfl_down_sync(0xffffffffu, ue, 1);
        float2 Gu[4];
        face_fwd2(us, ur, f2(us.y, ue), f2(ur.y, uer), Gu);
        if (add) {
            float2 e = z2;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float2 lo = add2(Gp[q], Gu[q]), hi = sub2(Gp[q], Gu[q]);
                e = fma2(mul2(fma2(Kl, cst.B2[q], cst.A2[q]), lo), lo, e);
                e = fma2(mul2(fma2(Kl, cst.B2[q + 4], cst.A2[q + 4]), hi), hi, e);
            }
            del = fma2(e, em, del);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) Gp[q] = Gu[q];
    };

    // stores of the owned outputs, predicated per row (no divergent branch)
    auto store_row = [&](bool on, int id, float xv, float rv, float pv) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %0, 0;\n\t"
            "@p st.global.f32 [%1], %4;\n\t@p st.global.f32 [%2], %5;\n\t@p st.global.f32 [%3], %6;\n\t}"
            ::"r"((int)on), "l"(x + id), "l"(r_out + id), "l"(p_out + id), "f"(xv), "f"(rv), "f"(pv)
            : "memory");
    };

    int st_issue = 0;
    for (int q = mbeg; q < mbeg + k4St - 1; ++q) {
        issue(q, st_issue);
        st_issue = st_issue + 1 == k4St ? 0 : st_issue + 1;
    }
    int st = 0;
    // Step m: stage A forms u_i, p_i at plane m; the face stage applies cell
    // layer m-1 to p (completing s at plane m-1) and adds the energies of
    // layer m-3 from u at planes m-3 and m-2; stage B forms r_{i+1}, u_{i+1}
    // at plane m-1 and writes the owned outputs.  In the steady part of the
    // march (STEADY) every stage is active, the planes are interior and the
    // loads are in range, so none of these conditions is evaluated.
    auto step = [&](const int m, auto steady_tag) {
        constexpr bool STEADY = decltype(steady_tag)::value;
        if (STEADY) {
            const int q = m + k4St - 1, pofs = NXY * q, cofs = CXY * q;
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const int R = R0 + b;
                const int id = nofs[b] + pofs, kid = kofs[b] + cofs;
                cp_async4n(&sm.ld_r[st_issue][R][tx], r + id, nsz[b]);
                if (!FIRST) cp_async4n(&sm.ld_p[st_issue][R][tx], p + id, nsz[b]);
                cp_async4n(&sm.ld_x[st_issue][R][tx], x + id, xsz[b]);
                cp_async4n(&sm.ld_k[st_issue][R][tx], K + kid, ksz[b]);
            }
            cp_async_commit();
        } else {
            issue(m + k4St - 1, st_issue);
        }
        st_issue = st_issue + 1 == k4St ? 0 : st_issue + 1;
        cp_async_wait_ring4();
        __syncthreads();
        const bool stageA = STEADY || m >= k0 - 1;
        const bool plane_live =
            STEADY || (m >= 0 && m < g.Nz && !(((dm & 16) && m == 0) || ((dm & 32) && m == g.Nz - 1)));
        // ---- stage A: u_i and p_i at plane m
        const float kk0 = sm.ld_k[st][R0][tx], kk1 = sm.ld_k[st][R0 + 1][tx], kk2 = sm.ld_k[st][Rext][tx];
        const float kd0 = __shfl_down_sync(0xffffffffu, kk0, 1);
        const float kd1 = __shfl_down_sync(0xffffffffu, kk1, 1);
        const float kd2 = __shfl_down_sync(0xffffffffu, kk2, 1);
        const float2 kA = add2(f2(kk0, kk1), f2(kd0, kd1));
        const float2 Sc = add2(kA, f2(kA.y, kk2 + kd2));
        const float2 Kc = f2(kd1, kd2);
        float2 di = z2, mk = z2;
        if (plane_live) {
            const float nzc = STEADY ? 2.0f : (float)cells_along(m, g.Nz);
            const float2 den = fma2(dk2, add2(S_prev, Sc), mul2(amn, f2(nzc, nzc)));
            di = mul2(lm, f2(rcp_approx(den.x), rcp_approx(den.y)));
            mk = lm;
        }
        const float2 rv = f2(sm.ld_r[st][R0][tx], sm.ld_r[st][R0 + 1][tx]);
        const float2 u = mul2(di, rv);
        const float2 pn = FIRST ? u : fma2(beta2, f2(sm.ld_p[st][R0][tx], sm.ld_p[st][R0 + 1][tx]), u);
        const float2 ax = f2(sm.ld_x[st][R0][tx], sm.ld_x[st][R0 + 1][tx]);
        S_prev = Sc;
        sm.pc0[ty][tx] = pn.x;
        __syncthreads();
        // ---- face stage: cell layer m-1 applied to p
        float2 u4[4];
        {
            const float pe = sm.pc0[tyn][tx];
            const float2 pr = shfl_down2(pn);
            const float per = __shfl_down_sync(0xffffffffu, pe, 1);
            float2 F[4], G[4];
            face_fwd2(pn, pr, f2(pn.y, pe), f2(pr.y, per), F);
            if (STEADY || (m >= k0 && m - 1 >= 0 && m - 1 < g.ncz)) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float2 lo = mul2(add2(Fp[q], F[q]), fma2(Kf1, cst.B2[q], cst.A2[q]));
                    const float2 hi = mul2(sub2(Fp[q], F[q]), fma2(Kf1, cst.B2[q + 4], cst.A2[q + 4]));
                    G[q] = fma2(add2(lo, hi), fm, Tp[q]);
                    if (stageA) Tp[q] = mul2(sub2(lo, hi), fm);
                }
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    G[q] = Tp[q];
                    if (stageA) Tp[q] = z2;
                }
            }
            face_bwd2(G, u4);
            if (stageA) {
#pragma unroll
                for (int q = 0; q < 4; ++q) Fp[q] = F[q];
            }
        }
        // energies of layer m-3 (u at plane m-2 from the previous stage B)
        if (STEADY) {
            energies(true, Kf3);
        } else if (m - 2 >= k0 && m - 2 <= k1 && m - 2 < g.Nz) {
            const int lc = m - 3;
            energies(lc >= k0 && lc < k1 && lc < g.ncz, Kf3);
        }
        sm.sc2[ty][tx] = u4[2].y;
        sm.sc3[ty][tx] = u4[3].y;
        __syncthreads();
        // ---- stage B: r_{i+1}, u_{i+1} at plane m-1; owned outputs
        const int kb = m - 1;
        if (STEADY || (kb >= k0 && kb <= k1 && kb < g.Nz)) {
            const float2 d2 = f2(sm.sc2[typ][tx], u4[2].x);
            const float2 d3 = f2(sm.sc3[typ][tx], u4[3].x);
            const float2 t = add2(u4[1], d3);
            const float2 sh = f2(__shfl_up_sync(0xffffffffu, t.x, 1), __shfl_up_sync(0xffffffffu, t.y, 1));
            const float2 sv = add2(add2(u4[0], d2), sh);
            const float2 rn = fma2(mul2(nalpha2, hm), sv, hr);
            const float2 un = mul2(hdi, rn);
            us = un;
            if (STEADY || kb < k1) {
                const float2 ro = mul2(rn, om);
                gam = fma2(ro, un, gam);
                rho = fma2(ro, rn, rho);
                const float2 xn = fma2(alpha2, hp, hx);
                const int ofs = NXY * kb;
                store_row(own[0], nofs[0] + ofs, xn.x, rn.x, hp.x);
                store_row(own[1], nofs[1] + ofs, xn.y, rn.y, hp.y);
            }
            sm.us0[ty][tx] = us.x;
        }
        if (stageA) {
            hr = rv;
            hp = pn;
            hdi = di;
            hm = mk;
            hx = ax;
        }
        Kf3 = Kf2;
        Kf2 = Kf1;
        Kf1 = Kc;
        st = st + 1 == k4St ? 0 : st + 1;
    };
    // steady steps: every stage active (m - 3 >= k0, m - 1 < k1), interior
    // planes, and the issued plane m + 5 inside both the mesh and the march
    const int ms0 = max(k0 + 3, mbeg), ms1 = min(k1 - 4, g.Nz - 7);
    int m = mbeg;
    for (; m < ms0 && m <= mend; ++m) step(m, std::false_type{});
    for (; m <= ms1; ++m) step(m, std::true_type{});
    for (; m <= mend; ++m) step(m, std::false_type{});
    {
        const int lc = k1 - 1;
        __syncthreads();
        if (lc >= k0 && lc < g.ncz) energies(true, Kf3);
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// the scalars of the next iteration from the reduced gamma, delta and rho
// (one thread): convergence, breakdown and non-finite checks
__device__ __forceinline__ void q1_cg_scalars(Scal* s, double gt, double dt_, double rt, int first) {
    s->rr = rt;
    if (!first) s->iters += 1;
    if (!isfinite(gt) || !isfinite(dt_) || !isfinite(rt)) {
        s->status = ST_NAN;
        s->done = 1;
    } else if (rt <= s->tol2 * s->bb || s->iters >= s->max_iter) {
        s->done = 1;
    } else {
        double a = 0.0, bta = 0.0;
        if (first) {
            a = gt / dt_;
        } else {
            bta = gt / s->rz;
            const double den = dt_ - bta * gt / s->alpha;
            a = gt / den;
            if (!(den > 0.0)) { s->status = ST_BREAKDOWN; s->done = 1; }
        }
        if (!(gt > 0.0) || !(dt_ > 0.0)) { s->status = ST_BREAKDOWN; s->done = 1; }
        s->alpha = a;
        s->beta = bta;
    }
    s->pq = dt_;
    s->rz = gt;
}

// One CG iteration over the whole mesh.  The CTAs form groups of ntx, one
// CTA per tile column of a tile row (bx = CTA % ntx), and the members of a
// group march the same node planes of the same tile row side by side, so
// that x-neighbouring tiles read their shared halos and write the sectors
// they share at about the same time (both stay in L2).  The tile rows, each
// Nz planes long, are laid end to end and group q takes planes
// [q R / Q, (q + 1) R / Q) of that sequence (R = nty x Nz, Q groups): every
// CTA has the same number of planes to march whatever the mesh.  The last
// CTA to finish reduces the partial sums.
template <bool FIRST>
__global__ void __launch_bounds__(kCgThreads, 1)
q1_cg_kernel(const Grid g, const float* __restrict__ K, float* __restrict__ x, const float* __restrict__ r,
             const float* __restrict__ p, float* __restrict__ r_out, float* __restrict__ p_out,
             const Q1HeadConst cst, const int ntx, const int nty, Scal* __restrict__ s, double* __restrict__ part,
             const int stride) {
    if (s->done) return;
    extern __shared__ __align__(16) unsigned char q1_smem_raw[];
    Q1Smem4& sm = *reinterpret_cast<Q1Smem4*>(q1_smem_raw);
    const float alpha = FIRST ? 0.0f : (float)s->alpha;
    const float beta = FIRST ? 0.0f : (float)s->beta;
    const int groups = gridDim.x / ntx;
    const int grp = blockIdx.x / ntx, bx = blockIdx.x % ntx;
    const long long R = (long long)nty * g.Nz;
    const long long f0 = R * grp / groups, f1 = R * (grp + 1) / groups;
    float2 gam = f2(0.0f, 0.0f), del = gam, rho = gam;
    for (long long f = f0; f < f1;) {
        const long long by = f / g.Nz;
        const int k0 = (int)(f - by * g.Nz);
        const long long rest = f1 - f;
        const int k1 = rest < (long long)(g.Nz - k0) ? k0 + (int)rest : g.Nz;
        q1_cg_tile2p<FIRST>(g, K, x, r, p, r_out, p_out, cst, bx, (int)by, ntx, nty, k0, k1, alpha, beta, sm, gam,
                            del, rho);
        f += k1 - k0;
    }
    double v[3];
    v[0] = block_sum_t(gam.x + gam.y);
    v[1] = block_sum_t(del.x + del.y);
    v[2] = block_sum_t(rho.x + rho.y);
    const unsigned nblk = gridDim.x;
    if (!publish_and_ticket(s, part, v, 3, stride, nblk)) return;
    const double gt = last_cta_sum(part, (int)nblk);
    const double dt_ = last_cta_sum(part + stride, (int)nblk);
    const double rt = last_cta_sum(part + 2 * (size_t)stride, (int)nblk);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        s->ticket = 0;
        q1_cg_scalars(s, gt, dt_, rt, FIRST);
    }
}

// ---------------------------------------------------------------------------
// Persistent CG over many Q1 problems (the batched inner head solves): one
// cooperative launch runs the first pass and up to `iters` iterations of
// every problem that has not converged.  Per iteration:
//   phase 1: the CTAs take the (problem, tile, z chunk) work items
//            round-robin, march each tile as the single-problem kernel does
//            and write the item's partial sums to its problem's slots;
//   barrier;
//   phase 2: CTA b forms the scalars of problems b, b + grid, ... (fixed
//            summation order, so the result is deterministic) and counts the
//            problems still running;
//   barrier; the launch ends once no problem is running.
// Converged problems drop out of the work list (their items are skipped).
// Every barrier wait is bounded: a wait that is not complete within `budget`
// clock cycles sets sync->err and the kernel returns; a CTA that sees
// sync->err set stops waiting at once.  The host turns sync->err into
// HT_ETIMEOUT.  drop_cta >= 0 makes that CTA leave at its first barrier
// without arriving, which lets a test make the other CTAs' waits run out.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool batch_barrier(Q1BatchSync* sync, unsigned nblk, long long budget, bool drop) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        int ok = 1;
        volatile unsigned* vgen = &sync->gen;
        volatile int* verr = &sync->err;
        const unsigned g0 = *vgen;
        __threadfence();   // release: this CTA's writes before its arrival
        if (drop) {
            ok = 0;
        } else if (atomicAdd(&sync->count, 1u) + 1u == nblk) {
            sync->count = 0;
            __threadfence();
            atomicAdd(&sync->gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*vgen == g0) {
                if (*verr) { ok = 0; break; }
                if (clock64() - t0 > budget) {
                    if (atomicExch(&sync->err, 1) == 0) sync->err_cta = (int)blockIdx.x;
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        ok_s = ok;
    }
    __syncthreads();
    __threadfence();   // acquire: later loads see what the other CTAs wrote before arriving
    return ok_s != 0;
}

__global__ void __launch_bounds__(kCgThreads, 1)
q1_cg_batch_kernel(const Q1BatchProb* __restrict__ probs, const int nprob, const int* __restrict__ item_prob,
                   const int nitems, const int iters, const long long budget, Q1BatchSync* __restrict__ sync,
                   const int drop_cta) {
    extern __shared__ __align__(16) unsigned char q1b_smem_raw[];
    Q1Smem4& sm = *reinterpret_cast<Q1Smem4*>(q1b_smem_raw);
    __shared__ Q1BatchProb P;
    __shared__ int skip_s, par_s;
    __shared__ float alpha_s, beta_s;
    const bool lead = threadIdx.x == 0 && threadIdx.y == 0;
    const unsigned nblk = gridDim.x;
    if (((volatile Q1BatchSync*)sync)->err) return;
    int running = 0;
    for (int it = 0; it <= iters; ++it) {
        const int first = it == 0;
        for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
            __syncthreads();   // the previous item is finished with P and the shared planes
            if (lead) {
                P = probs[item_prob[item]];
                const volatile Scal* vs = P.s;
                skip_s = vs->done;
                // pass j of a solve reads copy j % 2 of r and p (the first pass is pass 0)
                par_s = first ? 0 : ((vs->iters + 1) & 1);
                alpha_s = first ? 0.0f : (float)vs->alpha;
                beta_s = first ? 0.0f : (float)vs->beta;
            }
            __syncthreads();
            if (skip_s) continue;
            const int local = item - P.item0;
            const int bx = local % P.ntx, by = (local / P.ntx) % P.nty, bz = local / (P.ntx * P.nty);
            const int a = par_s;
            const int k0 = (int)((long long)bz * P.g.Nz / P.nzc), k1 = (int)((long long)(bz + 1) * P.g.Nz / P.nzc);
            float2 gam = f2(0.0f, 0.0f), del = gam, rho = gam;
            if (first)
                q1_cg_tile2p<true>(P.g, P.K, P.x, P.r[a], P.p[a], P.r[a ^ 1], P.p[a ^ 1], P.cst, bx, by, P.ntx,
                                   P.nty, k0, k1, alpha_s, beta_s, sm, gam, del, rho);
            else
                q1_cg_tile2p<false>(P.g, P.K, P.x, P.r[a], P.p[a], P.r[a ^ 1], P.p[a ^ 1], P.cst, bx, by, P.ntx,
                                    P.nty, k0, k1, alpha_s, beta_s, sm, gam, del, rho);
            double v[3];
            v[0] = block_sum_t(gam.x + gam.y);
            v[1] = block_sum_t(del.x + del.y);
            v[2] = block_sum_t(rho.x + rho.y);
            if (lead) {
                P.part[local] = v[0];
                P.part[(size_t)P.stride + local] = v[1];
                P.part[2 * (size_t)P.stride + local] = v[2];
            }
        }
        if (!batch_barrier(sync, nblk, budget, first && (int)blockIdx.x == drop_cta)) return;
        int cnt = 0;
        for (int pi = blockIdx.x; pi < nprob; pi += gridDim.x) {
            __syncthreads();
            if (lead) {
                P = probs[pi];
                skip_s = ((volatile Scal*)P.s)->done;
            }
            __syncthreads();
            if (skip_s) continue;
            const double gt = last_cta_sum(P.part, P.nitems);
            const double dt_ = last_cta_sum(P.part + P.stride, P.nitems);
            const double rt = last_cta_sum(P.part + 2 * (size_t)P.stride, P.nitems);
            if (lead) {
                q1_cg_scalars(P.s, gt, dt_, rt, first);
                cnt += P.s->done ? 0 : 1;
            }
        }
        if (lead) atomicAdd(&sync->active[it & 1], cnt);
        if (!batch_barrier(sync, nblk, budget, false)) return;
        running = ((volatile int*)sync->active)[it & 1];
        if (blockIdx.x == 0 && lead) sync->active[(it + 1) & 1] = 0;
        if (running == 0) break;
    }
    if (blockIdx.x == 0 && lead) sync->running = running;
}

// Eigenvalue parts of the Q1 cell operator in the h x h x h basis (see the
// file comment): lambda_l = A_l + K_c B_l with A_l = alpha M_l / 64 and
// B_l = dt K_l / 64, so that the kernel scales by the raw cell K.
Q1HeadConst q1_head_const(const double H[3], double alpha, double dt) {
    Q1HeadConst c{};
    double m1[3][2], k1[3][2];
    for (int d = 0; d < 3; ++d) {
        m1[d][0] = H[d];
        m1[d][1] = H[d] / 3.0;
        k1[d][0] = 0.0;
        k1[d][1] = 4.0 / H[d];
    }
    for (int cz = 0; cz < 2; ++cz)
        for (int by = 0; by < 2; ++by)
            for (int ax = 0; ax < 2; ++ax) {
                const int l = ax + 2 * by + 4 * cz;
                const double M = m1[0][ax] * m1[1][by] * m1[2][cz];
                const double Kl = k1[0][ax] * m1[1][by] * m1[2][cz] + m1[0][ax] * k1[1][by] * m1[2][cz] +
                                  m1[0][ax] * m1[1][by] * k1[2][cz];
                c.A[l] = (float)(alpha * M / 64.0);
                c.B[l] = (float)(dt * Kl / 64.0);
                c.A2[l] = make_float2(c.A[l], c.A[l]);
                c.B2[l] = make_float2(c.B[l], c.B[l]);
            }
    const double dM = H[0] * H[1] * H[2] / 27.0;
    const double dK = H[1] * H[2] / (9.0 * H[0]) + H[0] * H[2] / (9.0 * H[1]) + H[0] * H[1] / (9.0 * H[2]);
    c.am3 = (float)(alpha * dM);
    c.dk3 = (float)(dt * dK);
    return c;
}

int q1_split_z(int Nz, int tiles, int resident) {
    // chunks of node planes: waves of resident CTAs x (planes per chunk + 3
    // planes of pipeline start-up), ties to fewer chunks
    int best = 1;
    long long best_cost = -1;
    for (int z = 1; z <= Nz && z <= 64; ++z) {
        const long long waves = ((long long)tiles * z + resident - 1) / resident;
        const long long cost = waves * ((Nz + z - 1) / z + 3);
        if (best_cost < 0 || cost < best_cost) { best_cost = cost; best = z; }
    }
    return best;
}

// ---------------------------------------------------------------------------
// Heat operator on Q1 cells, fused into the BiCGStab iteration of the FP32
// inner heat solve (Eq. 4 in energy form):
//     A_T u = c_T M u + dt lambda K u + dt c_w C(q) u (+ dt d_w u on injection-well nodes),
//     C_ij = sum over Gauss points of W N_i (q . grad N_j),  q = -K_c grad h^{n+1}.
// Mass and conduction use the h x h x h eigenbasis of the head kernel.  The
// advection uses the structure of Q1 at the 2-point Gauss rule: du/dx is
// constant in x and bilinear in (y, z), so at the 8 Gauss points it takes 4
// values, the interpolation of the 4 x-edge differences of the cell by the
// 1D Gauss-point matrix B = [[g1, g0], [g0, g1]] (g0, g1 the two Gauss
// abscissae on [0, 1]) in y and z; the same holds for q from the x-edge
// differences of h.  Testing with N_i and summing the two x Gauss points
// (N_0 + N_1 = 1 there) leaves, for every node (a, b, c) of the cell,
//     dt c_w (-K_c) W [Rx(b,c) / Hx^2 + Ry(a,c) / Hy^2 + Rz(a,b) / Hz^2],
// Rx = B^T B^T applied to the Gauss-point products of the interpolated h and
// u differences (W = Hx Hy Hz / 8, the Gauss weight of the cell).
//
// Two launches per BiCGStab iteration, each one tiled march like the head
// kernel (halo of one node, tile of at most 30 x 22 node columns):
//   MODE 0: p' = r + beta (p - omega v), v' = A (D^-1 p'); the last CTA
//           forms alpha = rho / (r^.v');
//   MODE 1: s = r - alpha v', t = A (D^-1 s); the last CTA forms
//           omega = (t.s) / (t.t);
// then the pointwise update of x and r (fbi_update_kernel).  p and v are read
// on the halo and written on the tile, so they come in two copies (an
// iteration reads one and writes the other).
// ---------------------------------------------------------------------------
constexpr int kHTX = 30, kHTY = 22;          // largest owned tile of the heat kernel
constexpr int kHStages = 3;

struct Q1HeatConst {
    float MA[8], KB[8];     // mode eigenvalues: lambda_l = c_T MA_l + lambda KB_l
    float g0, g1;           // Gauss abscissae on [0, 1]
    float fx, fy, fz;       // dt c_w W / H_d^2 (times -K_c per cell)
    float cT, lam;          // uniform values (per-cell arrays when present)
    float dt;
};

struct Q1HeatSmem {
    float ld_r[kHStages][kSY][kSX];
    float ld_d[kHStages][kSY][kSX];
    float ld_h[kHStages][kSY][kSX];
    float ld_p[kHStages][kSY][kSX];
    float ld_v[kHStages][kSY][kSX];
    float ld_k[kHStages][kSY][kSX];
    float ld_o[kHStages][kSY][kSX];   // r^ (MODE 0) at owned nodes
    float ld_w[kHStages][kSY][kSX];   // injection-well coefficients at owned nodes
    float uc[kSY][kSX];               // operator input at the plane of stage A
    float hc[kSY][kSX];               // head at the plane of stage A
    float sc[4][kSY][kSX];            // corner contributions of each cell
};

// 2D interpolation of a 2 x 2 array d[j][i] (i fastest) to the Gauss points:
// o[qj][qi] = sum B[qj][j] B[qi][i] d[j][i], B[q][i] = g1 if q == i else g0
__device__ __forceinline__ void gauss2(const float (&d)[4], float g0, float g1, float (&o)[4]) {
    float t[4];
    t[0] = fmaf(g1, d[0], g0 * d[1]);   // along i
    t[1] = fmaf(g0, d[0], g1 * d[1]);
    t[2] = fmaf(g1, d[2], g0 * d[3]);
    t[3] = fmaf(g0, d[2], g1 * d[3]);
    o[0] = fmaf(g1, t[0], g0 * t[2]);   // along j
    o[1] = fmaf(g1, t[1], g0 * t[3]);
    o[2] = fmaf(g0, t[0], g1 * t[2]);
    o[3] = fmaf(g0, t[1], g1 * t[3]);
}

template <int MODE, bool PERCELL, bool WELLS>
__global__ void __launch_bounds__(kBX * kBY, 2)
q1_heat_kernel(const Grid g, const float* __restrict__ K, const float* __restrict__ cTc,
               const float* __restrict__ lamc, const float* __restrict__ h, const float* __restrict__ r,
               const float* __restrict__ Dinv, const float* __restrict__ p, const float* __restrict__ v,
               const float* __restrict__ rh, const float* __restrict__ wd, float* __restrict__ p_out,
               float* __restrict__ y_out, const Q1HeatConst cst, const int ntx, const int nty, const int nzc,
               Scal* __restrict__ s, double* __restrict__ part, const int stride) {
    if (s->done) return;
    extern __shared__ __align__(16) unsigned char q1h_smem_raw[];
    Q1HeatSmem& sm = *reinterpret_cast<Q1HeatSmem*>(q1h_smem_raw);
    const float beta = (float)s->beta, omega = (float)s->omega, alpha = (float)s->alpha;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i0 = (int)((long long)blockIdx.x * g.Nx / ntx), i1 = (int)((long long)(blockIdx.x + 1) * g.Nx / ntx);
    const int j0 = (int)((long long)blockIdx.y * g.Ny / nty), j1 = (int)((long long)(blockIdx.y + 1) * g.Ny / nty);
    const int k0 = (int)((long long)blockIdx.z * g.Nz / nzc), k1 = (int)((long long)(blockIdx.z + 1) * g.Nz / nzc);
    const int w = i1 - i0, hh = j1 - j0;
    const int NXY = g.Nx * g.Ny, CXY = g.ncx * g.ncy;
    const int dm = g.dmask;
    const int mbeg = k0 - 1, mend = k1;

    // slot (R, C) = node (C - 1, R - 1) of the tile and the cell whose low corner it is
    unsigned fl[kRows];
    int nxy[kRows], cxy[kRows];
#pragma unroll
    for (int b = 0; b < kRows; ++b) {
        const int R = ty + kBY * b, C = tx;
        const int gi = i0 + C - 1, gj = j0 + R - 1;
        unsigned f = 0;
        if (R >= 1 && R <= hh && C >= 1 && C <= w) f |= F_OWN;
        if (gi >= 0 && gi < g.Nx && gj >= 0 && gj < g.Ny) f |= F_NIN;
        if (gi >= 0 && gi < g.ncx && gj >= 0 && gj < g.ncy) f |= F_FIN;
        if (((dm & 1) && gi == 0) || ((dm & 2) && gi == g.Nx - 1) || ((dm & 4) && gj == 0) ||
            ((dm & 8) && gj == g.Ny - 1))
            f |= F_DXY;
        fl[b] = f;
        nxy[b] = (f & F_NIN) ? gi + g.Nx * gj : 0;
        cxy[b] = (f & F_FIN) ? gi + g.ncx * gj : 0;
    }

    auto issue = [&](int q) {
        if (q <= mend) {
            const int st = (q - mbeg) % kHStages;
            const bool plane_ok = q >= 0 && q < g.Nz;
            const bool layer_ok = q >= 0 && q < g.ncz;
            const int pofs = plane_ok ? NXY * q : 0, cofs = layer_ok ? CXY * q : 0;
#pragma unroll
            for (int b = 0; b < kRows; ++b) {
                const int R = ty + kBY * b, C = tx;
                const bool nok = plane_ok && (fl[b] & F_NIN);
                const int id = nok ? nxy[b] + pofs : 0;
                cp_async4(&sm.ld_r[st][R][C], r + id, nok);
                cp_async4(&sm.ld_d[st][R][C], Dinv + id, nok);
                cp_async4(&sm.ld_h[st][R][C], h + id, nok);
                cp_async4(&sm.ld_v[st][R][C], v + id, nok);
                if (MODE == 0) {
                    cp_async4(&sm.ld_p[st][R][C], p + id, nok);
                    cp_async4(&sm.ld_o[st][R][C], rh + id, nok && (fl[b] & F_OWN));
                }
                if (WELLS) cp_async4(&sm.ld_w[st][R][C], wd + id, nok && (fl[b] & F_OWN));
                const bool kok = layer_ok && (fl[b] & F_FIN);
                cp_async4(&sm.ld_k[st][R][C], K + (kok ? cxy[b] + cofs : 0), kok);
            }
        }
        cp_async_commit();
    };

    // per-row state carried up the march
    float hu[kRows], hv[kRows], hrh[kRows], hwd[kRows];   // node values of the plane of stage B
    float Up[kRows][4], Hp[kRows][4], Fp[kRows][4], Tp[kRows][4];
    float Kf[kRows], cTf[kRows], lamf[kRows];
#pragma unroll
    for (int b = 0; b < kRows; ++b) {
        hu[b] = hv[b] = hrh[b] = hwd[b] = 0.0f;
        Kf[b] = 0.0f;
        cTf[b] = cst.cT;
        lamf[b] = cst.lam;
#pragma unroll
        for (int q = 0; q < 4; ++q) Up[b][q] = Hp[b][q] = Fp[b][q] = Tp[b][q] = 0.0f;
    }
    float acc0 = 0.0f, acc1 = 0.0f;

    issue(mbeg);
    issue(mbeg + 1);
    for (int m = mbeg; m <= mend; ++m) {
        issue(m + 2);
        asm volatile("cp.async.wait_group 2;\n" ::: "memory");
        __syncthreads();
        const int st = (m - mbeg) % kHStages;
        const bool plane_ok = m >= 0 && m < g.Nz;
        const bool dirz = ((dm & 16) && m == 0) || ((dm & 32) && m == g.Nz - 1);
        // ---- stage A: the operator input at plane m
        float au[kRows], av[kRows], arh[kRows], awd[kRows], aK[kRows], acT[kRows], alam[kRows];
#pragma unroll
        for (int b = 0; b < kRows; ++b) {
            const int R = ty + kBY * b, C = tx;
            const float rv = sm.ld_r[st][R][C];
            const float vv = sm.ld_v[st][R][C];
            // MODE 0: p' = r + beta (p - omega v); MODE 1: s = r - alpha v
            const float val = MODE == 0 ? fmaf(beta, fmaf(-omega, vv, sm.ld_p[st][R][C]), rv) : fmaf(-alpha, vv, rv);
            const float uin = sm.ld_d[st][R][C] * val;
            const bool free_node = plane_ok && (fl[b] & F_NIN) && !(fl[b] & F_DXY) && !dirz;
            sm.uc[R][C] = free_node ? uin : 0.0f;
            sm.hc[R][C] = sm.ld_h[st][R][C];
            au[b] = uin;
            av[b] = val;
            arh[b] = MODE == 0 ? sm.ld_o[st][R][C] : 0.0f;
            awd[b] = WELLS ? sm.ld_w[st][R][C] : 0.0f;
            aK[b] = sm.ld_k[st][R][C];
            const int cid = cxy[b] + CXY * m;
            acT[b] = PERCELL && (fl[b] & F_FIN) && m >= 0 && m < g.ncz ? __ldg(cTc + cid) : cst.cT;
            alam[b] = PERCELL && (fl[b] & F_FIN) && m >= 0 && m < g.ncz ? __ldg(lamc + cid) : cst.lam;
        }
        __syncthreads();
        // ---- cell stage: cell layer m-1 (corners at planes m-1 and m)
        const bool lay_ok = m - 1 >= 0 && m - 1 < g.ncz && m >= k0;
#pragma unroll
        for (int b = 0; b < kRows; ++b) {
            const int R = ty + kBY * b, C = tx;
            const int R1 = R + 1 < kSY ? R + 1 : R, C1 = C + 1 < kSX ? C + 1 : C;
            float U[4] = {sm.uc[R][C], sm.uc[R][C1], sm.uc[R1][C], sm.uc[R1][C1]};
            float H[4] = {sm.hc[R][C], sm.hc[R][C1], sm.hc[R1][C], sm.hc[R1][C1]};
            float F[4];
            face_fwd(U[0], U[1], U[2], U[3], F);
            float bot[4] = {0.0f, 0.0f, 0.0f, 0.0f}, top[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            if (lay_ok && (fl[b] & F_FIN)) {
                // mass + conduction in the eigenbasis
                float lo[4], hi[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    lo[q] = (Fp[b][q] + F[q]) * fmaf(lamf[b], cst.KB[q], cTf[b] * cst.MA[q]);
                    hi[q] = (Fp[b][q] - F[q]) * fmaf(lamf[b], cst.KB[q + 4], cTf[b] * cst.MA[q + 4]);
                }
                float bh[4], th[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) { bh[q] = lo[q] + hi[q]; th[q] = lo[q] - hi[q]; }
                face_bwd(bh, bot);
                face_bwd(th, top);
                // advection: edge differences of u and h (corner index a + 2 b, plane c)
                const float* U0 = Up[b];
                const float* H0 = Hp[b];
                float du[4], dh[4], iu[4], ih[4], pr[4], rx[4], ry[4], rz[4];
                // x: differences along a at (b, c): index b + 2 c
                du[0] = U0[1] - U0[0]; du[1] = U0[3] - U0[2]; du[2] = U[1] - U[0]; du[3] = U[3] - U[2];
                dh[0] = H0[1] - H0[0]; dh[1] = H0[3] - H0[2]; dh[2] = H[1] - H[0]; dh[3] = H[3] - H[2];
                gauss2(du, cst.g0, cst.g1, iu);
                gauss2(dh, cst.g0, cst.g1, ih);
#pragma unroll
                for (int q = 0; q < 4; ++q) pr[q] = iu[q] * ih[q];
                gauss2(pr, cst.g0, cst.g1, rx);
                // y: differences along b at (a, c): index a + 2 c
                du[0] = U0[2] - U0[0]; du[1] = U0[3] - U0[1]; du[2] = U[2] - U[0]; du[3] = U[3] - U[1];
                dh[0] = H0[2] - H0[0]; dh[1] = H0[3] - H0[1]; dh[2] = H[2] - H[0]; dh[3] = H[3] - H[1];
                gauss2(du, cst.g0, cst.g1, iu);
                gauss2(dh, cst.g0, cst.g1, ih);
#pragma unroll
                for (int q = 0; q < 4; ++q) pr[q] = iu[q] * ih[q];
                gauss2(pr, cst.g0, cst.g1, ry);
                // z: differences along c at (a, b): index a + 2 b
#pragma unroll
                for (int q = 0; q < 4; ++q) { du[q] = U[q] - U0[q]; dh[q] = H[q] - H0[q]; }
                gauss2(du, cst.g0, cst.g1, iu);
                gauss2(dh, cst.g0, cst.g1, ih);
#pragma unroll
                for (int q = 0; q < 4; ++q) pr[q] = iu[q] * ih[q];
                gauss2(pr, cst.g0, cst.g1, rz);
                const float mk = -Kf[b];
                const float fx = mk * cst.fx, fy = mk * cst.fy, fz = mk * cst.fz;
                // node (a, b, c): fx Rx(b, c) + fy Ry(a, c) + fz Rz(a, b)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int a = q & 1, bb = q >> 1;
                    bot[q] += fmaf(fx, rx[bb], fmaf(fy, ry[a], fz * rz[q]));
                    top[q] += fmaf(fx, rx[bb + 2], fmaf(fy, ry[a + 2], fz * rz[q]));
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                sm.sc[q][R][C] = Tp[b][q] + bot[q];
                Tp[b][q] = top[q];
                Fp[b][q] = F[q];
                Up[b][q] = U[q];
                Hp[b][q] = H[q];
            }
        }
        __syncthreads();
        // ---- stage B: owned nodes of plane m-1
        const int kb = m - 1;
        if (kb >= k0 && kb < k1) {
            const bool dirb = ((dm & 16) && kb == 0) || ((dm & 32) && kb == g.Nz - 1);
#pragma unroll
            for (int b = 0; b < kRows; ++b) {
                const int R = ty + kBY * b, C = tx;
                if (fl[b] & F_OWN) {
                    const int Rm = R > 0 ? R - 1 : 0, Cm = C > 0 ? C - 1 : 0;
                    float yv = (sm.sc[0][R][C] + sm.sc[1][R][Cm]) + (sm.sc[2][Rm][C] + sm.sc[3][Rm][Cm]);
                    if (WELLS) yv = fmaf(cst.dt * hwd[b], hu[b], yv);
                    const bool dir = (fl[b] & F_DXY) || dirb;
                    if (dir) yv = hu[b];
                    const int id = nxy[b] + NXY * kb;
                    y_out[id] = yv;
                    if (MODE == 0) {
                        p_out[id] = hv[b];
                        acc0 = fmaf(hrh[b], yv, acc0);
                    } else {
                        acc0 = fmaf(yv, hv[b], acc0);
                        acc1 = fmaf(yv, yv, acc1);
                    }
                }
            }
        }
#pragma unroll
        for (int b = 0; b < kRows; ++b) {
            hu[b] = au[b];
            hv[b] = av[b];
            hrh[b] = arh[b];
            hwd[b] = awd[b];
            Kf[b] = aK[b];
            cTf[b] = acT[b];
            lamf[b] = alam[b];
        }
    }
    double vals[2];
    vals[0] = block_sum_t(acc0);
    vals[1] = MODE == 1 ? block_sum_t(acc1) : 0.0;
    const unsigned nblk = gridDim.x * gridDim.y * gridDim.z;
    if (MODE == 0) {
        if (!publish_and_ticket(s, part, vals, 1, stride, nblk)) return;
        const double a = last_cta_sum(part, (int)nblk);
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            s->ticket = 0;
            s->rv = a;
            if (a == 0.0 || !isfinite(a)) { s->status = ST_BREAKDOWN; s->done = 1; }
            else s->alpha = s->rho / a;
        }
    } else {
        if (!publish_and_ticket(s, part + stride, vals, 2, stride, nblk)) return;
        const double a = last_cta_sum(part + stride, (int)nblk);
        const double b2 = last_cta_sum(part + 2 * (size_t)stride, (int)nblk);
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            s->ticket = 0;
            s->ts = a;
            s->tt = b2;
            s->omega = b2 == 0.0 ? 0.0 : a / b2;   // s = 0 exactly: x += alpha ph is the solution
        }
    }
}

Q1HeatConst q1_heat_const(const ht_ctx* c, double dt) {
    Q1HeatConst k{};
    const double* H = c->H;
    double m1[3][2], k1[3][2];
    for (int d = 0; d < 3; ++d) {
        m1[d][0] = H[d];
        m1[d][1] = H[d] / 3.0;
        k1[d][0] = 0.0;
        k1[d][1] = 4.0 / H[d];
    }
    for (int cz = 0; cz < 2; ++cz)
        for (int by = 0; by < 2; ++by)
            for (int ax = 0; ax < 2; ++ax) {
                const int l = ax + 2 * by + 4 * cz;
                const double M = m1[0][ax] * m1[1][by] * m1[2][cz];
                const double Kl = k1[0][ax] * m1[1][by] * m1[2][cz] + m1[0][ax] * k1[1][by] * m1[2][cz] +
                                  m1[0][ax] * m1[1][by] * k1[2][cz];
                k.MA[l] = (float)(M / 64.0);
                k.KB[l] = (float)(dt * Kl / 64.0);
            }
    const double d = 0.5 / sqrt(3.0);
    k.g0 = (float)(0.5 - d);
    k.g1 = (float)(0.5 + d);
    const double W = H[0] * H[1] * H[2] / 8.0;
    k.fx = (float)(dt * c->cw * W / (H[0] * H[0]));
    k.fy = (float)(dt * c->cw * W / (H[1] * H[1]));
    k.fz = (float)(dt * c->cw * W / (H[2] * H[2]));
    k.cT = (float)c->cT_u;
    k.lam = (float)c->lam_u;
    k.dt = (float)dt;
    return k;
}

template <int MODE, bool PERCELL, bool WELLS>
int launch_q1_heat(ht_ctx* c, const Grid& g, const Q1HeatConst& k, const float* r, const float* Dinv, const float* p,
                   const float* v, const float* rh, float* p_out, float* y_out, Scal* sc) {
    auto kern = q1_heat_kernel<MODE, PERCELL, WELLS>;
    static int resident = 0;
    const size_t smem = sizeof(Q1HeatSmem);
    if (resident == 0) {
        HT_CUDA(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int vv = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&vv, kern, kBX * kBY, smem) != cudaSuccess || vv < 1) vv = 1;
        resident = vv;
    }
    const int ntx = (g.Nx + kHTX - 1) / kHTX, nty = (g.Ny + kHTY - 1) / kHTY;
    const int sms = c->num_sms > 0 ? c->num_sms : 148;
    int nzc = c->opts.z_chunks > 0 ? std::min(c->opts.z_chunks, g.Nz) : q1_split_z(g.Nz, ntx * nty, resident * sms);
    while (nzc > 1 && ntx * nty * nzc > c->part_stride) --nzc;
    if (ntx * nty * nzc > c->part_stride) return fail(c, HT_EINVAL, "too many partial sums");
    kern<<<dim3(ntx, nty, nzc), dim3(kBX, kBY), smem, c->stream>>>(
        g, c->K32, c->cT32, c->lam32, c->h32, r, Dinv, p, v, rh, c->wdn32, p_out, y_out, k, ntx, nty, nzc, sc,
        c->part, c->part_stride);
    ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    return HT_OK;
}

template <int MODE>
int launch_q1_heat_any(ht_ctx* c, const Grid& g, const Q1HeatConst& k, const float* r, const float* Dinv,
                       const float* p, const float* v, const float* rh, float* p_out, float* y_out, Scal* sc) {
    const bool percell = c->cT32 != nullptr || c->lam32 != nullptr;
    const bool wells = c->wdn32 != nullptr;
    if (percell && (c->cT32 == nullptr || c->lam32 == nullptr))
        return fail(c, HT_EINVAL, "per-cell c_T and lambda must be given together for the single-pass heat kernel");
    if (percell)
        return wells ? launch_q1_heat<MODE, true, true>(c, g, k, r, Dinv, p, v, rh, p_out, y_out, sc)
                     : launch_q1_heat<MODE, true, false>(c, g, k, r, Dinv, p, v, rh, p_out, y_out, sc);
    return wells ? launch_q1_heat<MODE, false, true>(c, g, k, r, Dinv, p, v, rh, p_out, y_out, sc)
                 : launch_q1_heat<MODE, false, false>(c, g, k, r, Dinv, p, v, rh, p_out, y_out, sc);
}

}  // namespace

bool q1_cg_available(const ht_ctx* c, int fp32) {
    return fp32 && c->grid.P == 1 && c->K32 != nullptr && !c->graded &&
           (c->opts.apply_variant == HT_APPLY_AUTO || c->opts.apply_variant == HT_APPLY_SINGLE_PASS);
}

bool q1_bicgstab_available(const ht_ctx* c) {
    const bool percell_ok = (c->cT32 == nullptr) == (c->lam32 == nullptr);
    return c->grid.P == 1 && c->K32 != nullptr && c->h32 != nullptr && percell_ok && c->n_dint == 0 && !c->graded &&
           (c->opts.apply_variant == HT_APPLY_AUTO || c->opts.apply_variant == HT_APPLY_SINGLE_PASS);
}

int q1_bicgstab_iteration32(ht_ctx* c, float dt, float* x, float* r, const float* rh, const float* p_in,
                            const float* v_in, float* p_out, float* v_out, float* t, const float* Dinv, Scal* sc) {
    Grid g = c->grid;
    g.dmask = c->dmask[HT_TEMP];
    const Q1HeatConst k = q1_heat_const(c, (double)dt);
    HT_TRY(launch_q1_heat_any<0>(c, g, k, r, Dinv, p_in, v_in, rh, p_out, v_out, sc));
    HT_TRY(launch_q1_heat_any<1>(c, g, k, r, Dinv, nullptr, v_out, nullptr, nullptr, t, sc));
    return launch_fbi_update32(c, x, r, p_out, v_out, t, Dinv, rh, sc);
}

int q1_batch_prepare(Q1Batch& q, ht_ctx* const* probs, int n, double dt, int planes, cudaStream_t st,
                     std::string* err) {
    auto bad = [&](int code, const char* msg) {
        if (err) *err = msg;
        return code;
    };
    int dev = 0, sms = 0, resident = 0;
    const size_t smem = sizeof(Q1Smem4);
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaFuncSetAttribute(q1_cg_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, q1_cg_batch_kernel, kCgThreads, smem) != cudaSuccess ||
        resident < 1)
        return bad(HT_ECUDA, "persistent batch kernel: occupancy query failed");
    const int slots = resident * sms;
    // tiles of every problem, then the z chunking: the same number of node
    // planes per chunk for all problems, chosen to minimise (waves of items
    // over the co-resident CTAs) x (planes per chunk + 3 planes of start-up)
    std::vector<int> ntx(n), nty(n), Nz(n);
    for (int i = 0; i < n; ++i) {
        const ht_ctx* c = probs[i];
        if (!q1_cg_available(c, 1)) return bad(HT_EINVAL, "persistent batch needs Q1 problems with the single-pass kernels");
        ntx[i] = (c->grid.Nx + k4TX - 1) / k4TX;
        nty[i] = (c->grid.Ny + k4TY - 1) / k4TY;
        Nz[i] = c->grid.Nz;
    }
    auto count_items = [&](int L, std::vector<int>* nzc) {
        long long items = 0;
        for (int i = 0; i < n; ++i) {
            const int z = std::max(1, (Nz[i] + L - 1) / L);
            if (nzc) (*nzc)[i] = z;
            items += (long long)ntx[i] * nty[i] * z;
        }
        return items;
    };
    int best = planes;
    if (best <= 0) {
        long long best_cost = -1;
        int maxNz = *std::max_element(Nz.begin(), Nz.end());
        for (int L = 2; L <= maxNz; ++L) {
            const long long waves = (count_items(L, nullptr) + slots - 1) / slots;
            const long long cost = waves * (L + 3);
            if (best_cost < 0 || cost < best_cost) { best_cost = cost; best = L; }
        }
        if (best_cost < 0) best = std::max(1, maxNz);
    }
    std::vector<int> nzc(n);
    const long long total = count_items(best, &nzc);
    if (total > (1LL << 30)) return bad(HT_EINVAL, "persistent batch: too many work items");
    std::vector<Q1BatchProb> h(n);
    std::vector<int> items;
    items.reserve((size_t)total);
    for (int i = 0; i < n; ++i) {
        ht_ctx* c = probs[i];
        Q1BatchProb& P = h[i];
        memset(&P, 0, sizeof(P));
        P.g = c->grid;
        P.g.dmask = c->dmask[HT_HEAD];
        P.K = c->K32;
        P.x = c->d32;
        P.r[0] = c->r32;
        P.r[1] = c->s32;
        P.p[0] = c->p32;
        P.p[1] = c->q32;
        P.cst = q1_head_const(c->H, c->Ss, dt);
        P.ntx = ntx[i];
        P.nty = nty[i];
        P.nzc = nzc[i];
        P.item0 = (int)items.size();
        P.nitems = ntx[i] * nty[i] * nzc[i];
        if (P.nitems > c->part_stride) return bad(HT_EINVAL, "persistent batch: too many partial sums for a problem");
        P.part = c->part;
        P.stride = c->part_stride;
        P.s = c->scal + 1;
        for (int k = 0; k < P.nitems; ++k) items.push_back(i);
    }
    // buffers grow only; descriptors are uploaded on every call (the
    // operator scalars and vectors of a problem may change between steps)
    if (n > q.cap_probs || (int)items.size() > q.cap_items || !q.d_sync) {
        q1_batch_free(q);
        if (cudaMalloc(&q.d_probs, n * sizeof(Q1BatchProb)) != cudaSuccess ||
            cudaMalloc(&q.d_items, items.size() * sizeof(int)) != cudaSuccess ||
            cudaMalloc(&q.d_sync, sizeof(Q1BatchSync)) != cudaSuccess ||
            cudaMallocHost(&q.h_sync, sizeof(Q1BatchSync)) != cudaSuccess) {
            q1_batch_free(q);
            return bad(HT_ENOMEM, "persistent batch: allocation failed");
        }
        q.cap_probs = n;
        q.cap_items = (int)items.size();
    }
    if (cudaMemcpyAsync(q.d_probs, h.data(), n * sizeof(Q1BatchProb), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(q.d_items, items.data(), items.size() * sizeof(int), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        q1_batch_free(q);
        return bad(HT_ECUDA, "persistent batch: descriptor upload failed");
    }
    q.nprob = n;
    q.nitems = (int)items.size();
    q.grid = (int)std::min<long long>(slots, q.nitems);
    q.planes = best;
    q.dt = dt;
    return HT_OK;
}

int q1_batch_run(Q1Batch& q, cudaStream_t st, int max_iter, long long budget, int drop_cta, int* running,
                 int* err_cta, std::string* err) {
    auto bad = [&](int code, const char* msg) {
        if (err) *err = msg;
        return code;
    };
    *running = 0;
    *err_cta = -1;
    if (!q.d_probs || q.nitems < 1) return bad(HT_EINVAL, "persistent batch: not prepared");
    if (cudaMemsetAsync(q.d_sync, 0, sizeof(Q1BatchSync), st) != cudaSuccess)
        return bad(HT_ECUDA, "persistent batch: barrier reset failed");
    const Q1BatchProb* probs = (const Q1BatchProb*)q.d_probs;
    const int* items = q.d_items;
    int nprob = q.nprob, nitems = q.nitems, iters = std::max(0, max_iter);
    long long bud = budget;
    Q1BatchSync* sync = (Q1BatchSync*)q.d_sync;
    int drop = drop_cta;
    void* args[] = {(void*)&probs, (void*)&nprob, (void*)&items, (void*)&nitems, (void*)&iters,
                    (void*)&bud, (void*)&sync, (void*)&drop};
    // cooperative: every CTA of the grid is resident at once, which the
    // grid barrier needs
    if (cudaLaunchCooperativeKernel((const void*)q1_cg_batch_kernel, dim3(q.grid), dim3(32, kCgBY), args,
                                    sizeof(Q1Smem4), st) != cudaSuccess)
        return bad(HT_ECUDA, "persistent batch: cooperative launch failed");
    if (cudaMemcpyAsync(q.h_sync, q.d_sync, sizeof(Q1BatchSync), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return bad(HT_ECUDA, "persistent batch: status readback failed");
    const Q1BatchSync* hs = (const Q1BatchSync*)q.h_sync;
    if (hs->err) {
        *err_cta = hs->err_cta;
        return bad(HT_ETIMEOUT, "persistent batch: a grid-barrier wait ran out of its budget");
    }
    *running = hs->running;
    return HT_OK;
}

void q1_batch_free(Q1Batch& q) {
    if (q.d_probs) cudaFree(q.d_probs);
    if (q.d_items) cudaFree(q.d_items);
    if (q.d_sync) cudaFree(q.d_sync);
    if (q.h_sync) cudaFreeHost(q.h_sync);
    q.d_probs = nullptr;
    q.d_items = nullptr;
    q.d_sync = nullptr;
    q.h_sync = nullptr;
    q.nprob = q.nitems = q.grid = q.cap_probs = q.cap_items = 0;
    q.dt = -1.0;
}

int q1_cg_iteration32(ht_ctx* c, float dt, float* x, const float* r, const float* p, float* r_out, float* p_out,
                      Scal* sc, int first) {
    Grid g = c->grid;
    g.dmask = c->dmask[HT_HEAD];
    const Q1HeadConst cst = q1_head_const(c->H, c->Ss, (double)dt);
    const int ntx = (g.Nx + k4TX - 1) / k4TX, nty = (g.Ny + k4TY - 1) / k4TY;
    static int resident = 0;
    const size_t smem = sizeof(Q1Smem4);
    if (resident == 0) {
        HT_CUDA(c, cudaFuncSetAttribute(q1_cg_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        HT_CUDA(c, cudaFuncSetAttribute(q1_cg_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, q1_cg_kernel<false>, kCgThreads, smem) != cudaSuccess ||
            v < 1)
            v = 1;
        resident = v;
    }
    const int sms = c->num_sms > 0 ? c->num_sms : 148;
    // groups of ntx CTAs (one per tile column of a tile row), as many groups
    // as fit in the co-resident slots, at least 8 node planes per group (each
    // z segment repeats 3 planes of pipeline start-up); z_chunks > 0 asks
    // for about that many segments per tile row instead
    const long long R = (long long)nty * g.Nz;
    long long Q = c->opts.z_chunks > 0 ? (long long)nty * std::min(c->opts.z_chunks, g.Nz)
                                       : std::min<long long>(std::max(1, resident * sms / ntx), (R + 7) / 8);
    Q = std::max(1LL, std::min({Q, R, (long long)(c->part_stride / ntx)}));
    if (Q * ntx > c->part_stride) return fail(c, HT_EINVAL, "too many partial sums");
    const dim3 grid((unsigned)(Q * ntx)), block(32, kCgBY);
    if (first)
        q1_cg_kernel<true><<<grid, block, smem, c->stream>>>(g, c->K32, x, r, p, r_out, p_out, cst, ntx, nty, sc,
                                                             c->part, c->part_stride);
    else
        q1_cg_kernel<false><<<grid, block, smem, c->stream>>>(g, c->K32, x, r, p, r_out, p_out, cst, ntx, nty, sc,
                                                              c->part, c->part_stride);
    ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    return HT_OK;
}

}  // namespace ht
