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

#include <algorithm>

#include "ht_device.cuh"
#include "ht_internal.cuh"

namespace ht {
namespace {

constexpr int kTX = 28, kTY = 20;   // largest owned tile (node columns)
constexpr int kBX = 32, kBY = 8;    // threads: lanes along x, warps along y
constexpr int kRows = 3;            // rows of a thread: (kTY + 4) / kBY
constexpr int kSX = 32, kSY = 24;   // shared plane: kRows * kBY rows of 32
constexpr int kStages = 6;          // load ring (five planes in flight)

struct Q1HeadConst {
    float A[8], B[8];   // lambda_l = A_l + (dt K_c) B_l, mode l = a + 2 b + 4 c
    float am3;          // alpha * diag(M_e)
    float dk3;          // dt * diag(K_e)
};

struct Q1Smem {
    float ld_r[kStages][kSY][kSX];
    float ld_p[kStages][kSY][kSX];
    float ld_x[kStages][kSY][kSX];
    float ld_k[kStages][kSY][kSX];
    float pc[kSY][kSX];        // p_i at the plane of stage A
    float sc[4][kSY][kSX];     // corner contributions of each face to s
    float us[kSY][kSX];        // u_{i+1} at the plane of stage B
};

__device__ __forceinline__ void cp_async4(float* sdst, const float* gsrc, bool valid) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    const int n = valid ? 4 : 0;   // 0: no bytes are read, the word is zero-filled
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gsrc), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_ring() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(kStages - 1) : "memory");
}

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

__global__ void __launch_bounds__(kBX * kBY, 2)
q1_cg_kernel(const Grid g, const float* __restrict__ K, float* __restrict__ x, const float* __restrict__ r,
             const float* __restrict__ p, float* __restrict__ r_out, float* __restrict__ p_out,
             const Q1HeadConst cst, const int ntx, const int nty, const int nzc, Scal* __restrict__ s,
             double* __restrict__ part, const int stride, const int first) {
    if (s->done) return;
    extern __shared__ __align__(16) unsigned char q1_smem_raw[];
    Q1Smem& sm = *reinterpret_cast<Q1Smem*>(q1_smem_raw);
    const float alpha = first ? 0.0f : (float)s->alpha;
    const float beta = first ? 0.0f : (float)s->beta;
    const int tx = threadIdx.x, ty = threadIdx.y;
    // owned tile and chunk (balanced splits)
    const int i0 = (int)((long long)blockIdx.x * g.Nx / ntx), i1 = (int)((long long)(blockIdx.x + 1) * g.Nx / ntx);
    const int j0 = (int)((long long)blockIdx.y * g.Ny / nty), j1 = (int)((long long)(blockIdx.y + 1) * g.Ny / nty);
    const int k0 = (int)((long long)blockIdx.z * g.Nz / nzc), k1 = (int)((long long)(blockIdx.z + 1) * g.Nz / nzc);
    const int w = i1 - i0, h = j1 - j0;
    const int NXY = g.Nx * g.Ny, CXY = g.ncx * g.ncy;
    const int dm = g.dmask;
    const int mbeg = k0 - 2, mend = k1 + 1;

    // slot (R, C) = (ty + 8 b, tx) holds node (C - 1, R - 1) of the tile, the
    // face (cell column) whose low corner that node is, and the cell column
    // (C - 2, R - 2) of the K plane
    unsigned fl[kRows];
    int nxy[kRows], cxy[kRows];
    float ncxy[kRows];
#pragma unroll
    for (int b = 0; b < kRows; ++b) {
        const int R = ty + kBY * b, C = tx;
        const int gi = i0 + C - 1, gj = j0 + R - 1;
        unsigned f = 0;
        if (R >= 1 && R <= h && C >= 1 && C <= w) f |= F_OWN;
        if (R >= 1 && R < h + 2 && C >= 1 && C < w + 2) f |= F_R1;
        if (gi >= 0 && gi < g.Nx && gj >= 0 && gj < g.Ny) f |= F_NIN;
        if (gi >= 0 && gi < g.ncx && gj >= 0 && gj < g.ncy) f |= F_FIN;
        if (gi - 1 >= 0 && gi - 1 < g.ncx && gj - 1 >= 0 && gj - 1 < g.ncy) f |= F_KIN;
        if (((dm & 1) && gi == 0) || ((dm & 2) && gi == g.Nx - 1) || ((dm & 4) && gj == 0) ||
            ((dm & 8) && gj == g.Ny - 1))
            f |= F_DXY;
        fl[b] = f;
        nxy[b] = (f & F_NIN) ? gi + g.Nx * gj : 0;
        cxy[b] = (f & F_KIN) ? (gi - 1) + g.ncx * (gj - 1) : 0;
        ncxy[b] = (float)(cells_along(gi, g.Nx) * cells_along(gj, g.Ny));
    }

    // loads of plane / cell layer q into ring slot (q - mbeg) % kStages; every
    // slot of the 32 x 24 planes is written (zero where outside the mesh)
    auto issue = [&](int q) {
        if (q <= mend) {
            const int st = (q - mbeg) % kStages;
            const bool plane_ok = q >= 0 && q < g.Nz;
            const bool layer_ok = q >= 0 && q < g.ncz;
            const int pofs = plane_ok ? NXY * q : 0, cofs = layer_ok ? CXY * q : 0;
#pragma unroll
            for (int b = 0; b < kRows; ++b) {
                const int R = ty + kBY * b, C = tx;
                const bool nok = plane_ok && (fl[b] & F_NIN);
                const int id = nok ? nxy[b] + pofs : 0;
                cp_async4(&sm.ld_r[st][R][C], r + id, nok);
                if (!first) cp_async4(&sm.ld_p[st][R][C], p + id, nok);
                cp_async4(&sm.ld_x[st][R][C], x + id, nok && (fl[b] & F_OWN));
                const bool kok = layer_ok && (fl[b] & F_KIN);
                cp_async4(&sm.ld_k[st][R][C], K + (kok ? cxy[b] + cofs : 0), kok);
            }
        }
        cp_async_commit();
    };

    // per-row state carried up the march
    float S_prev[kRows];                                 // sum of the node's 4 cell K, layer below
    float hr[kRows], hp[kRows], hdi[kRows], hx[kRows];   // node values of the plane of stage B
    float Fp[kRows][4], Tp[kRows][4], Gp[kRows][4];      // face transforms of p and u, top parts
    float Kf1[kRows], Kf2[kRows], Kf3[kRows];            // the face's K one, two, three layers down
#pragma unroll
    for (int b = 0; b < kRows; ++b) {
        S_prev[b] = 0.0f;
        hr[b] = hp[b] = hdi[b] = hx[b] = 0.0f;
        Kf1[b] = Kf2[b] = Kf3[b] = 0.0f;
#pragma unroll
        for (int q = 0; q < 4; ++q) Fp[b][q] = Tp[b][q] = Gp[b][q] = 0.0f;
    }
    float gam = 0.0f, rho = 0.0f, del = 0.0f;

    for (int q = mbeg; q < mbeg + kStages - 1; ++q) issue(q);
    // Step m: stage A forms u_i, p_i at plane m; the face stage applies cell
    // layer m-1 to p (completing s at plane m-1) and adds the energies of
    // layer m-3 from u at planes m-3 and m-2; stage B forms r_{i+1}, u_{i+1}
    // at plane m-1 and writes the owned outputs.
    for (int m = mbeg; m <= mend; ++m) {
        issue(m + kStages - 1);
        cp_async_wait_ring();
        __syncthreads();
        const int st = (m - mbeg) % kStages;
        const bool stageA = m >= k0 - 1;
        const bool plane_ok = m >= 0 && m < g.Nz;
        const bool dirz = ((dm & 16) && m == 0) || ((dm & 32) && m == g.Nz - 1);
        const float nz_cells = (float)cells_along(m, g.Nz);
        // ---- stage A
        float ar[kRows], ap[kRows], adi[kRows], ax[kRows], Kc[kRows];
#pragma unroll
        for (int b = 0; b < kRows; ++b) {
            const int R = ty + kBY * b, C = tx;
            const int R1 = R + 1 < kSY ? R + 1 : R, C1 = C + 1 < kSX ? C + 1 : C;
            const float Sc = (sm.ld_k[st][R][C] + sm.ld_k[st][R][C1]) + (sm.ld_k[st][R1][C] + sm.ld_k[st][R1][C1]);
            Kc[b] = sm.ld_k[st][R1][C1];
            const bool live = plane_ok && (fl[b] & F_NIN) && !(fl[b] & F_DXY) && !dirz;
            const float di = live ? __frcp_rn(fmaf(cst.dk3, S_prev[b] + Sc, cst.am3 * ncxy[b] * nz_cells)) : 0.0f;
            const float rv = sm.ld_r[st][R][C];
            const float pv = first ? 0.0f : sm.ld_p[st][R][C];
            const float pn = fmaf(beta, pv, di * rv);
            sm.pc[R][C] = pn;
            ar[b] = rv;
            ap[b] = pn;
            adi[b] = di;
            ax[b] = sm.ld_x[st][R][C];
            S_prev[b] = Sc;
        }
        __syncthreads();
        // ---- face stage
        const bool apply_on = m >= k0;
        const bool lay_ok = m - 1 >= 0 && m - 1 < g.ncz;
        const int lc = m - 3;                 // layer of the energies
        const bool energy_on = lc >= k0 && lc < k1 && lc < g.ncz;
#pragma unroll
        for (int b = 0; b < kRows; ++b) {
            const int R = ty + kBY * b, C = tx;
            const int R1 = R + 1 < kSY ? R + 1 : R, C1 = C + 1 < kSX ? C + 1 : C;
            const bool cell = apply_on && lay_ok && (fl[b] & F_FIN);
            float F[4];
            face_fwd(sm.pc[R][C], sm.pc[R][C1], sm.pc[R1][C], sm.pc[R1][C1], F);
            float G[4], u[4], top[4];
            const float bk = Kf1[b];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float lo = (Fp[b][q] + F[q]) * fmaf(bk, cst.B[q], cst.A[q]);
                const float hi = (Fp[b][q] - F[q]) * fmaf(bk, cst.B[q + 4], cst.A[q + 4]);
                G[q] = cell ? Tp[b][q] + (lo + hi) : Tp[b][q];
                top[q] = cell ? lo - hi : 0.0f;
            }
            face_bwd(G, u);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                sm.sc[q][R][C] = u[q];
                if (stageA) {
                    Tp[b][q] = top[q];
                    Fp[b][q] = F[q];
                }
            }
            // energies of layer m-3: u at plane m-2 is still in us (stage B of
            // the previous step), its transform at plane m-3 in Gp
            if (m - 2 >= k0 && m - 2 <= k1 && m - 2 < g.Nz) {
                float Gu[4];
                face_fwd(sm.us[R][C], sm.us[R][C1], sm.us[R1][C], sm.us[R1][C1], Gu);
                if (energy_on && (fl[b] & F_OWN) && (fl[b] & F_FIN)) {
                    const float ek = Kf3[b];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float lo = Gp[b][q] + Gu[q], hi = Gp[b][q] - Gu[q];
                        del = fmaf(fmaf(ek, cst.B[q], cst.A[q]) * lo, lo, del);
                        del = fmaf(fmaf(ek, cst.B[q + 4], cst.A[q + 4]) * hi, hi, del);
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) Gp[b][q] = Gu[q];
            }
        }
        __syncthreads();
        // ---- stage B
        const int kb = m - 1;
        const bool stageB = kb >= k0 && kb <= k1 && kb < g.Nz;
        const bool owned_plane = kb < k1;
        if (stageB) {
#pragma unroll
            for (int b = 0; b < kRows; ++b) {
                const int R = ty + kBY * b, C = tx;
                const int Rm = R > 0 ? R - 1 : 0, Cm = C > 0 ? C - 1 : 0;
                const float sv = (sm.sc[0][R][C] + sm.sc[1][R][Cm]) + (sm.sc[2][Rm][C] + sm.sc[3][Rm][Cm]);
                const float rn = hdi[b] != 0.0f ? fmaf(-alpha, sv, hr[b]) : hr[b];
                const float un = hdi[b] * rn;
                sm.us[R][C] = un;
                if (owned_plane && (fl[b] & F_OWN)) {
                    const int id = nxy[b] + NXY * kb;
                    x[id] = fmaf(alpha, hp[b], hx[b]);
                    r_out[id] = rn;
                    p_out[id] = hp[b];
                    gam = fmaf(rn, un, gam);
                    rho = fmaf(rn, rn, rho);
                }
            }
        }
        // histories move up one plane
#pragma unroll
        for (int b = 0; b < kRows; ++b) {
            if (stageA) {
                hr[b] = ar[b];
                hp[b] = ap[b];
                hdi[b] = adi[b];
                hx[b] = ax[b];
            }
            Kf3[b] = Kf2[b];
            Kf2[b] = Kf1[b];
            Kf1[b] = Kc[b];
        }
    }
    // the march ends with stage B at plane k1; the energies of layer k1 - 1
    // need u at planes k1 - 1 and k1, both in hand after the last step
    {
        const int lc = k1 - 1;
        if (lc >= k0 && lc < g.ncz) {
            __syncthreads();
#pragma unroll
            for (int b = 0; b < kRows; ++b) {
                const int R = ty + kBY * b, C = tx;
                const int R1 = R + 1 < kSY ? R + 1 : R, C1 = C + 1 < kSX ? C + 1 : C;
                float Gu[4];
                face_fwd(sm.us[R][C], sm.us[R][C1], sm.us[R1][C], sm.us[R1][C1], Gu);
                if ((fl[b] & F_OWN) && (fl[b] & F_FIN)) {
                    const float ek = Kf3[b];   // K of layer k1 - 1 after the last shift
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float lo = Gp[b][q] + Gu[q], hi = Gp[b][q] - Gu[q];
                        del = fmaf(fmaf(ek, cst.B[q], cst.A[q]) * lo, lo, del);
                        del = fmaf(fmaf(ek, cst.B[q + 4], cst.A[q + 4]) * hi, hi, del);
                    }
                }
            }
        }
    }
    double v[3];
    v[0] = block_sum_t(gam);
    v[1] = block_sum_t(del);
    v[2] = block_sum_t(rho);
    const unsigned nblk = gridDim.x * gridDim.y * gridDim.z;
    if (!publish_and_ticket(s, part, v, 3, stride, nblk)) return;
    const double gt = last_cta_sum(part, (int)nblk);
    const double dt_ = last_cta_sum(part + stride, (int)nblk);
    const double rt = last_cta_sum(part + 2 * (size_t)stride, (int)nblk);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        s->ticket = 0;
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

}  // namespace

bool q1_cg_available(const ht_ctx* c, int fp32) {
    return fp32 && c->grid.P == 1 && c->K32 != nullptr &&
           (c->opts.apply_variant == HT_APPLY_AUTO || c->opts.apply_variant == HT_APPLY_SINGLE_PASS);
}

int q1_cg_iteration32(ht_ctx* c, float dt, float* x, const float* r, const float* p, float* r_out, float* p_out,
                      Scal* sc, int first) {
    Grid g = c->grid;
    g.dmask = c->dmask[HT_HEAD];
    const Q1HeadConst cst = q1_head_const(c->H, c->Ss, (double)dt);
    const int ntx = (g.Nx + kTX - 1) / kTX, nty = (g.Ny + kTY - 1) / kTY;
    static int resident = 0;
    const size_t smem = sizeof(Q1Smem);
    if (resident == 0) {
        HT_CUDA(c, cudaFuncSetAttribute(q1_cg_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, q1_cg_kernel, kBX * kBY, smem) != cudaSuccess || v < 1)
            v = 1;
        resident = v;
    }
    const int sms = c->num_sms > 0 ? c->num_sms : 148;
    int nzc = c->opts.z_chunks > 0 ? std::min(c->opts.z_chunks, g.Nz) : q1_split_z(g.Nz, ntx * nty, resident * sms);
    while (nzc > 1 && ntx * nty * nzc > c->part_stride) --nzc;
    if (ntx * nty * nzc > c->part_stride) return fail(c, HT_EINVAL, "too many partial sums");
    q1_cg_kernel<<<dim3(ntx, nty, nzc), dim3(kBX, kBY), smem, c->stream>>>(
        g, c->K32, x, r, p, r_out, p_out, cst, ntx, nty, nzc, sc, c->part, c->part_stride, first);
    ++c->n_launch;
    HT_CUDA(c, cudaGetLastError());
    return HT_OK;
}

}  // namespace ht
