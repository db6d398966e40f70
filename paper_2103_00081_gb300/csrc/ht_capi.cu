// C ABI of the hydrothermal step (include/ht.h): context set-up, host-side
// load tables, the time stepper and parity hooks.
#include <cuda_runtime.h>
#include <limits.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <vector>

#include "ht_internal.cuh"

namespace ht {

int fail(ht_ctx* c, int code, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

namespace {

thread_local std::string g_create_error;

// ---- 1D reference data --------------------------------------------------------
void gauss01(int n, double* x, double* w) {
    if (n == 2) {
        const double d = 0.5 / sqrt(3.0);
        x[0] = 0.5 - d; x[1] = 0.5 + d;
        w[0] = w[1] = 0.5;
    } else {
        const double d = 0.5 * sqrt(0.6);
        x[0] = 0.5 - d; x[1] = 0.5; x[2] = 0.5 + d;
        w[0] = 5.0 / 18.0; w[1] = 8.0 / 18.0; w[2] = 5.0 / 18.0;
    }
}

// Lagrange basis on the equispaced nodes {0, 1/P, ..., 1}
double lag(int P, int a, double xi) {
    double v = 1.0;
    for (int m = 0; m <= P; ++m)
        if (m != a) v *= (xi - (double)m / P) / ((double)(a - m) / P);
    return v;
}

double dlag(int P, int a, double xi) {
    double s = 0.0;
    for (int m = 0; m <= P; ++m) {
        if (m == a) continue;
        double t = 1.0 / ((double)(a - m) / P);
        for (int k = 0; k <= P; ++k)
            if (k != a && k != m) t *= (xi - (double)k / P) / ((double)(a - k) / P);
        s += t;
    }
    return s;
}

// cyclic Jacobi eigen-decomposition of a symmetric n x n matrix (n <= 3):
// A = U diag(lam) U^T, columns of U are eigenvectors
void jacobi_eig(int n, double A[3][3], double U[3][3], double lam[3]) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) U[i][j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += A[p][q] * A[p][q];
        if (off < 1e-300) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                if (A[p][q] == 0.0) continue;
                const double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
                for (int k = 0; k < n; ++k) {  // A = J^T A J
                    const double akp = A[k][p], akq = A[k][q];
                    A[k][p] = cs * akp - sn * akq;
                    A[k][q] = sn * akp + cs * akq;
                }
                for (int k = 0; k < n; ++k) {
                    const double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = cs * apk - sn * aqk;
                    A[q][k] = sn * apk + cs * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double ukp = U[k][p], ukq = U[k][q];
                    U[k][p] = cs * ukp - sn * ukq;
                    U[k][q] = sn * ukp + cs * ukq;
                }
            }
    }
    for (int i = 0; i < n; ++i) lam[i] = A[i][i];
}

// 1D element mass / stiffness on [0, H] and their fast-diagonalisation
// factors G (m = G^T G, k = G^T diag(lam) G).
void element_1d(int P, double H, double m[3][3], double k[3][3], double G[3][3], double lam[3]) {
    const int n = P + 1;
    double xq[3], wq[3];
    gauss01(n, xq, wq);
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) {
            double sm = 0, sk = 0;
            for (int q = 0; q < n; ++q) {
                sm += wq[q] * lag(P, a, xq[q]) * lag(P, b, xq[q]);
                sk += wq[q] * dlag(P, a, xq[q]) * dlag(P, b, xq[q]);
            }
            m[a][b] = H * sm;
            k[a][b] = sk / H;
        }
    // Cholesky m = L L^T
    double L[3][3] = {{0}};
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = m[i][j];
            for (int l = 0; l < j; ++l) s -= L[i][l] * L[j][l];
            L[i][j] = (i == j) ? sqrt(s) : s / L[j][j];
        }
    // Linv
    double Li[3][3] = {{0}};
    for (int i = 0; i < n; ++i) {
        Li[i][i] = 1.0 / L[i][i];
        for (int j = 0; j < i; ++j) {
            double s = 0;
            for (int l = j; l < i; ++l) s -= L[i][l] * Li[l][j];
            Li[i][j] = s / L[i][i];
        }
    }
    // C = Li k Li^T
    double C[3][3] = {{0}};
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double s = 0;
            for (int a = 0; a < n; ++a)
                for (int b = 0; b < n; ++b) s += Li[i][a] * k[a][b] * Li[j][b];
            C[i][j] = s;
        }
    double U[3][3];
    jacobi_eig(n, C, U, lam);
    // G = U^T L^T : G[i][j] = sum_l U[l][i] L[j][l]
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) G[i][j] = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double s = 0;
            for (int l = 0; l < n; ++l) s += U[l][i] * L[j][l];
            G[i][j] = s;
        }
}

void build_elem(ht_ctx* c) {
    const int P = c->grid.P, n = P + 1;
    ht::Elem<double>& e = c->e64;
    memset(&e, 0, sizeof(e));
    // a graded mesh takes the constants of the unit cube; its kernels scale
    // them per cell (volume, 1/h per axis)
    const double unit[3] = {1.0, 1.0, 1.0};
    const double* H = c->graded ? unit : c->H;
    double m[3][3][3], k[3][3][3];
    for (int d = 0; d < 3; ++d) element_1d(P, H[d], m[d], k[d], e.G[d], e.Lam[d]);
    double xq[3], wq[3];
    gauss01(n, xq, wq);
    for (int q = 0; q < n; ++q)
        for (int a = 0; a < n; ++a) {
            e.B[q][a] = lag(P, a, xq[q]);
            e.D[q][a] = dlag(P, a, xq[q]);
        }
    const double vol = H[0] * H[1] * H[2];
    for (int qz = 0; qz < n; ++qz)
        for (int qy = 0; qy < n; ++qy)
            for (int qx = 0; qx < n; ++qx) e.W[qx + n * (qy + n * qz)] = wq[qx] * wq[qy] * wq[qz] * vol;
    for (int d = 0; d < 3; ++d) e.invH[d] = 1.0 / H[d];
    for (int a = 0; a < n; ++a) {
        e.dm1[a] = m[0][a][a];
        e.dk1[a] = k[0][a][a];
    }
    for (int cc = 0; cc < n; ++cc)
        for (int b = 0; b < n; ++b)
            for (int a = 0; a < n; ++a) {
                const int l = a + n * (b + n * cc);
                e.dM[l] = m[0][a][a] * m[1][b][b] * m[2][cc][cc];
                e.dK[l] = k[0][a][a] * m[1][b][b] * m[2][cc][cc] + m[0][a][a] * k[1][b][b] * m[2][cc][cc] +
                          m[0][a][a] * m[1][b][b] * k[2][cc][cc];
                e.LS[l] = e.Lam[0][a] + e.Lam[1][b] + e.Lam[2][cc];
            }
    // FP32 copy
    ht::Elem<float>& f = c->e32;
    const double* src = reinterpret_cast<const double*>(&e);
    float* dst = reinterpret_cast<float*>(&f);
    static_assert(sizeof(ht::Elem<double>) == 2 * sizeof(ht::Elem<float>), "Elem layout");
    for (size_t i = 0; i < sizeof(e) / sizeof(double); ++i) dst[i] = (float)src[i];
    // float-float copy: hi = nearest float, lo = nearest float to the remainder
    ht::df64* dd = reinterpret_cast<ht::df64*>(&c->edf);
    static_assert(sizeof(ht::Elem<double>) == sizeof(ht::Elem<ht::df64>), "Elem layout");
    for (size_t i = 0; i < sizeof(e) / sizeof(double); ++i) {
        const float hi = (float)src[i];
        dd[i] = ht::df64(hi, (float)(src[i] - (double)hi));
    }
}

// Head-operator constants of a cell of size H (fast-diagonalisation factors,
// eigenvalues and element diagonals) computed into a caller-owned struct; used
// by the allocation-free entry point, which has no context.
void head_elem_stack(int P, const double H[3], ht::Elem<double>& e) {
    const int n = P + 1;
    memset(&e, 0, sizeof(e));
    double m[3][3][3], k[3][3][3];
    for (int d = 0; d < 3; ++d) element_1d(P, H[d], m[d], k[d], e.G[d], e.Lam[d]);
    for (int cc = 0; cc < n; ++cc)
        for (int b = 0; b < n; ++b)
            for (int a = 0; a < n; ++a) {
                const int l = a + n * (b + n * cc);
                e.dM[l] = m[0][a][a] * m[1][b][b] * m[2][cc][cc];
                e.dK[l] = k[0][a][a] * m[1][b][b] * m[2][cc][cc] + m[0][a][a] * k[1][b][b] * m[2][cc][cc] +
                          m[0][a][a] * m[1][b][b] * k[2][cc][cc];
                e.LS[l] = e.Lam[0][a] + e.Lam[1][b] + e.Lam[2][cc];
            }
    for (int d = 0; d < 3; ++d) e.invH[d] = 1.0 / H[d];
}

// integral of phi_a over [0,1] (exact Gauss)
double phi_int(int P, int a) {
    double xq[3], wq[3];
    gauss01(P + 1, xq, wq);
    double s = 0;
    for (int q = 0; q <= P; ++q) s += wq[q] * lag(P, a, xq[q]);
    return s;
}

// integral of phi_a phi_b over [0,1] (exact Gauss)
double phi_phi_int(int P, int a, int b) {
    double xq[3], wq[3];
    gauss01(P + 1, xq, wq);
    double s = 0;
    for (int q = 0; q <= P; ++q) s += wq[q] * lag(P, a, xq[q]) * lag(P, b, xq[q]);
    return s;
}

// 1D boundary integral weight of node i along a direction with nc cells of size H
double node_int_1d(int P, int nc, double H, int i) {
    double s = 0;
    if (i % P == 0) {
        const int cl = i / P - 1, cr = i / P;
        if (cl >= 0) s += H * phi_int(P, P);
        if (cr < nc) s += H * phi_int(P, 0);
    } else {
        s += H * phi_int(P, i % P);
    }
    return s;
}

int axis_cells(const ht_ctx* c, int d);
// the same along axis d of the context (per-cell widths on a graded mesh)
double node_int_axis(const ht_ctx* c, int d, int i) {
    const int P = c->grid.P, nc = axis_cells(c, d);
    if (!c->graded) return node_int_1d(P, nc, c->H[d], i);
    double s = 0;
    if (i % P == 0) {
        const int cl = i / P - 1, cr = i / P;
        if (cl >= 0) s += c->widths[d][cl] * phi_int(P, P);
        if (cr < nc) s += c->widths[d][cr] * phi_int(P, 0);
    } else {
        s += c->widths[d][i / P] * phi_int(P, i % P);
    }
    return s;
}

template <typename T>
int dalloc(ht_ctx* c, T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T) + 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, HT_ENOMEM, "cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
    }
    *p = static_cast<T*>(q);
    return HT_OK;
}

template <typename T>
void dfree(T*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

// ---- geometry along an axis (uniform cells of size H, or the tensor-product
// widths of a graded mesh, Fig. 10b) ----------------------------------------
double axis_origin(const ht_ctx* c, int d) { return d == 0 ? c->mesh.x0 : (d == 1 ? c->mesh.y0 : c->mesh.z0); }
int axis_cells(const ht_ctx* c, int d) { return d == 0 ? c->mesh.nx : (d == 1 ? c->mesh.ny : c->mesh.nz); }
// low face of cell layer k along d, and its width
double face_at(const ht_ctx* c, int d, int k) {
    return c->graded ? c->faces[d][k] : axis_origin(c, d) + k * c->H[d];
}
double width_at(const ht_ctx* c, int d, int k) { return c->graded ? c->widths[d][k] : c->H[d]; }
// cell layer along d holding coordinate v (clamped to the mesh) and the local
// coordinate of v in it
void locate(const ht_ctx* c, int d, double v, int* ci, double* xi) {
    const int n = axis_cells(c, d);
    if (!c->graded) {
        const double s = (v - axis_origin(c, d)) / c->H[d];
        int k = (int)floor(s);
        k = std::max(0, std::min(k, n - 1));
        *ci = k;
        *xi = s - k;
        return;
    }
    const std::vector<double>& f = c->faces[d];
    int k = (int)(std::upper_bound(f.begin(), f.end(), v) - f.begin()) - 1;
    k = std::max(0, std::min(k, n - 1));
    *ci = k;
    *xi = (v - f[k]) / c->widths[d][k];
}
// coordinate of node i along d
double node_coord(const ht_ctx* c, int d, int i) {
    const int P = c->grid.P;
    if (!c->graded) return axis_origin(c, d) + i * (c->H[d] / P);
    const int k = std::min(i / P, axis_cells(c, d) - 1);
    return c->faces[d][k] + (i - P * k) * c->widths[d][k] / P;
}

// Vertical segment weights w_i = int_{z_bot}^{z_top} N_i(x, y, z) dz
int line_weights(ht_ctx* c, double x, double y, double ztop, double zbot, std::map<long long, double>& out,
                 const char* what) {
    const ht_mesh& m = c->mesh;
    const int P = c->grid.P;
    const double eps = 1e-9 * std::max(m.Lx, std::max(m.Ly, m.Lz));
    if (!(x >= m.x0 - eps && x <= m.x0 + m.Lx + eps && y >= m.y0 - eps && y <= m.y0 + m.Ly + eps))
        return fail(c, HT_EINVAL, "%s at (%g, %g) lies outside the box", what, x, y);
    if (!(ztop > zbot)) return fail(c, HT_EINVAL, "%s needs z_top > z_bot", what);
    const double lo = std::max(zbot, m.z0), hi = std::min(ztop, m.z0 + m.Lz);
    if (!(hi > lo)) return fail(c, HT_EINVAL, "%s segment does not intersect the box", what);
    int cxy[2];
    double fx[2][3];
    const double pos[2] = {x, y}, org[2] = {m.x0, m.y0};
    const int ncs[2] = {m.nx, m.ny};
    (void)org;
    (void)ncs;
    for (int d = 0; d < 2; ++d) {
        int ci = 0;
        double xi = 0.0;
        locate(c, d, pos[d], &ci, &xi);
        cxy[d] = ci;
        for (int a = 0; a <= P; ++a) fx[d][a] = lag(P, a, xi);
    }
    double xq[3], wq[3];
    gauss01(3, xq, wq);
    int cz0 = 0;
    if (!c->graded) {
        cz0 = (int)floor((lo - m.z0) / c->H[2]);
        cz0 = std::max(0, std::min(cz0, m.nz - 1));
    }
    for (int cz = cz0; cz < m.nz; ++cz) {
        const double Hz = width_at(c, 2, cz);
        const double a0 = face_at(c, 2, cz), a1 = c->graded ? c->faces[2][cz + 1] : a0 + Hz;
        if (a0 >= hi) break;
        const double s0 = std::max(a0, lo), s1 = std::min(a1, hi);
        if (s1 <= s0) continue;
        for (int cc = 0; cc <= P; ++cc) {
            double Iz = 0;
            for (int g = 0; g < 3; ++g) {
                const double zz = s0 + (s1 - s0) * xq[g];
                Iz += wq[g] * (s1 - s0) * lag(P, cc, (zz - a0) / Hz);
            }
            for (int b = 0; b <= P; ++b)
                for (int a = 0; a <= P; ++a) {
                    const long long i = (long long)P * cxy[0] + a, j = (long long)P * cxy[1] + b,
                                    k = (long long)P * cz + cc;
                    const long long id = i + (long long)c->grid.Nx * (j + (long long)c->grid.Ny * k);
                    out[id] += fx[0][a] * fx[1][b] * Iz;
                }
        }
    }
    return HT_OK;
}

// Cell-face index nearest to v along axis d (ties upwards), clamped to [0, n].
int snap_face(const ht_ctx* c, int d, double v) {
    const double org[3] = {c->mesh.x0, c->mesh.y0, c->mesh.z0};
    const int n[3] = {c->mesh.nx, c->mesh.ny, c->mesh.nz};
    if (c->graded) {   // the nearest face; of equally near faces the higher one
        const std::vector<double>& f = c->faces[d];
        int best = 0;
        for (int k = 1; k <= n[d]; ++k)
            if (fabs(f[k] - v) <= fabs(f[best] - v)) best = k;
        return best;
    }
    const double f = floor((v - org[d]) / c->H[d] + 0.5);
    return (int)std::max(0.0, std::min(f, (double)n[d]));
}

// Box source weights w_i = int_R N_i dS over the snapped rectangle R: on each
// cell face inside R the integral factors into Hx int phi_a * Hy int phi_b.
int box_weights(ht_ctx* c, const ht_box_src& b, std::map<long long, double>& out) {
    const int P = c->grid.P;
    const int i0 = snap_face(c, 0, b.x0), i1 = snap_face(c, 0, b.x1);
    const int j0 = snap_face(c, 1, b.y0), j1 = snap_face(c, 1, b.y1);
    const int k = snap_face(c, 2, b.z);
    if (i1 <= i0 || j1 <= j0) return fail(c, HT_EINVAL, "box source is empty once snapped to cell faces");
    double ix[3], iy[3];
    const long long kk = (long long)P * k;
    for (int cy = j0; cy < j1; ++cy)
        for (int cx = i0; cx < i1; ++cx) {
            for (int a = 0; a <= P; ++a) {
                ix[a] = width_at(c, 0, cx) * phi_int(P, a);
                iy[a] = width_at(c, 1, cy) * phi_int(P, a);
            }
            for (int bb = 0; bb <= P; ++bb)
                for (int a = 0; a <= P; ++a) {
                    const long long i = (long long)P * cx + a, j = (long long)P * cy + bb;
                    out[i + (long long)c->grid.Nx * (j + (long long)c->grid.Ny * kk)] += ix[a] * iy[bb];
                }
        }
    return HT_OK;
}

bool node_on_dirichlet_face(const ht_ctx* c, int field, long long id) {
    const Grid& g = c->grid;
    const int i = (int)(id % g.Nx), j = (int)((id / g.Nx) % g.Ny), k = (int)(id / ((long long)g.Nx * g.Ny));
    const int m = c->dmask[field];
    return ((m & 1) && i == 0) || ((m & 2) && i == g.Nx - 1) || ((m & 4) && j == 0) ||
           ((m & 8) && j == g.Ny - 1) || ((m & 16) && k == 0) || ((m & 32) && k == g.Nz - 1);
}

bool node_on_dirichlet(const ht_ctx* c, int field, long long id) {
    if (node_on_dirichlet_face(c, field, id)) return true;
    return field == HT_TEMP && std::binary_search(c->dint_host.begin(), c->dint_host.end(), id);
}

// Nodes held at a pile's temperature (Section 3.3): the nodes within the
// radius of the pile axis (lateral distance) whose z lies in the pile's
// depth range, or, when no node is that close, the node column nearest the
// axis (ties to the lower j, then the lower i) over the same depth range.
// Node coordinates are origin + index * H / P, compared with a tolerance of
// 1e-9 of the largest extent.  row = x, y, z_top, z_bot, radius, ...
int pile_surface_nodes(ht_ctx* c, const double* row, std::vector<long long>& out) {
    const Grid& g = c->grid;
    const ht_mesh& m = c->mesh;
    const double hx = c->H[0] / g.P, hy = c->H[1] / g.P;
    const double eps = 1e-9 * std::max(m.Lx, std::max(m.Ly, m.Lz));
    const double zlo = std::min(row[2], row[3]) - eps, zhi = std::max(row[2], row[3]) + eps;
    std::vector<int> ks;
    for (int k = 0; k < g.Nz; ++k) {
        const double z = node_coord(c, 2, k);
        if (z >= zlo && z <= zhi) ks.push_back(k);
    }
    out.clear();
    if (ks.empty()) return fail(c, HT_EINVAL, "pile surface (%g, %g) lies outside the mesh", row[0], row[1]);
    auto lat = [&](int i, int j) {
        const double dx = node_coord(c, 0, i) - row[0], dy = node_coord(c, 1, j) - row[1];
        return dx * dx + dy * dy;
    };
    const double r2 = row[4] * row[4] + eps;
    const double R = sqrt(r2);
    int i0 = 0, i1 = g.Nx - 1, j0 = 0, j1 = g.Ny - 1;   // a graded mesh scans every column
    if (!c->graded) {
        i0 = std::max(0, (int)floor((row[0] - R - m.x0) / hx) - 1);
        i1 = std::min(g.Nx - 1, (int)ceil((row[0] + R - m.x0) / hx) + 1);
        j0 = std::max(0, (int)floor((row[1] - R - m.y0) / hy) - 1);
        j1 = std::min(g.Ny - 1, (int)ceil((row[1] + R - m.y0) / hy) + 1);
    }
    std::vector<std::pair<int, int>> cols;
    for (int j = j0; j <= j1; ++j)
        for (int i = i0; i <= i1; ++i)
            if (lat(i, j) <= r2) cols.push_back({i, j});
    if (cols.empty()) {
        int bi = 0, bj = 0;
        double best = -1.0;
        for (int j = 0; j < g.Ny; ++j)
            for (int i = 0; i < g.Nx; ++i) {
                const double d = lat(i, j);
                if (best < 0.0 || d < best) { best = d; bi = i; bj = j; }
            }
        cols.push_back({bi, bj});
    }
    for (int k : ks)
        for (auto& ij : cols) out.push_back(ij.first + (long long)g.Nx * (ij.second + (long long)g.Ny * k));
    std::sort(out.begin(), out.end());
    return HT_OK;
}

// device tables of the pile-surface nodes and the heat Dirichlet rows off
// the faces (after the face masks are known)
int setup_pile_temperatures(ht_ctx* c) {
    dfree(c->ptemp_node); dfree(c->ptemp_pile); dfree(c->d_ptemp); dfree(c->dint);
    dfree(c->dint_a64); dfree(c->dint_b64); dfree(c->dint_a32);
    c->n_ptemp_nodes = 0;
    c->n_dint = 0;
    c->dint_host.clear();
    const int np = (int)(c->ptemp_rows.size() / 9);
    if (np == 0) return HT_OK;
    std::map<long long, int> owner;   // node -> the last pile that holds it
    std::vector<long long> nodes;
    for (int p = 0; p < np; ++p) {
        HT_TRY(pile_surface_nodes(c, &c->ptemp_rows[9 * (size_t)p], nodes));
        for (long long id : nodes) owner[id] = p;
    }
    std::vector<long long> nd;
    std::vector<int> pl;
    std::vector<double> prm(4 * (size_t)np);
    for (int p = 0; p < np; ++p)
        for (int q = 0; q < 4; ++q) prm[4 * (size_t)p + q] = c->ptemp_rows[9 * (size_t)p + 5 + q];
    for (auto& kv : owner) {
        nd.push_back(kv.first);
        pl.push_back(kv.second);
        if (!node_on_dirichlet_face(c, HT_TEMP, kv.first)) c->dint_host.push_back(kv.first);
    }
    const size_t nn = (size_t)c->grid.nn;
    c->n_ptemp_nodes = (int)nd.size();
    c->n_dint = (int)c->dint_host.size();
    if (cudaMalloc(&c->ptemp_node, nd.size() * sizeof(long long)) != cudaSuccess ||
        cudaMalloc(&c->ptemp_pile, pl.size() * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&c->d_ptemp, prm.size() * sizeof(double)) != cudaSuccess ||
        (c->n_dint > 0 && (cudaMalloc(&c->dint, c->dint_host.size() * sizeof(long long)) != cudaSuccess ||
                           cudaMalloc(&c->dint_a64, nn * sizeof(double)) != cudaSuccess ||
                           cudaMalloc(&c->dint_b64, nn * sizeof(double)) != cudaSuccess ||
                           cudaMalloc(&c->dint_a32, nn * sizeof(float)) != cudaSuccess))) {
        c->n_ptemp_nodes = c->n_dint = 0;
        return fail(c, HT_ENOMEM, "pile-surface tables: allocation failed");
    }
    HT_CUDA(c, cudaMemcpyAsync(c->ptemp_node, nd.data(), nd.size() * sizeof(long long), cudaMemcpyHostToDevice,
                               c->stream));
    HT_CUDA(c, cudaMemcpyAsync(c->ptemp_pile, pl.data(), pl.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    HT_CUDA(c, cudaMemcpyAsync(c->d_ptemp, prm.data(), prm.size() * sizeof(double), cudaMemcpyHostToDevice,
                               c->stream));
    if (c->n_dint > 0)
        HT_CUDA(c, cudaMemcpyAsync(c->dint, c->dint_host.data(), c->dint_host.size() * sizeof(long long),
                                   cudaMemcpyHostToDevice, c->stream));
    HT_CUDA(c, cudaStreamSynchronize(c->stream));
    return HT_OK;
}

// n-point Gauss-Legendre rule on [0, 1]: Newton iteration on the Legendre
// polynomial P_n from the standard cosine initial guesses.
void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double t = cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = t;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (t * p1 - p0) / (t * t - 1.0);
            const double dt = p1 / dp;
            t -= dt;
            if (fabs(dt) < 1e-16) break;
        }
        x[i] = 0.5 * (1.0 - t);
        w[i] = 1.0 / ((1.0 - t * t) * dp * dp);   // (2 / ((1-t^2) P'^2)) / 2
    }
}

// Source weights of a well: line weights (sigma = 0) or, for a lateral normal
// density of standard deviation sigma, w_i = Ix(cx,a) Iy(cy,b) Jz(cz,c) with
// the lateral cell integrals by a 10-point Gauss rule within 10 sigma.
int well_weights(ht_ctx* c, const ht_well& wl, std::map<long long, double>& out) {
    if (!(wl.sigma > 0)) return line_weights(c, wl.x, wl.y, wl.z_top, wl.z_bot, out, "well");
    std::map<long long, double> probe;
    HT_TRY(line_weights(c, wl.x, wl.y, wl.z_top, wl.z_bot, probe, "well"));   // validates the segment
    const ht_mesh& m = c->mesh;
    const int P = c->grid.P;
    std::vector<double> xg, wg;
    gauss_legendre01(10, xg, wg);
    std::vector<std::pair<std::pair<int, int>, double>> I[2];
    const double centre[2] = {wl.x, wl.y}, org[2] = {m.x0, m.y0};
    const int ncs[2] = {m.nx, m.ny};
    const double sg = wl.sigma;
    for (int d = 0; d < 2; ++d) {
        (void)org;
        for (int ci = 0; ci < ncs[d]; ++ci) {
            const double H = width_at(c, d, ci);
            const double a0 = face_at(c, d, ci);
            if (a0 > centre[d] + 10 * sg || a0 + H < centre[d] - 10 * sg) continue;
            for (int a = 0; a <= P; ++a) {
                double sum = 0.0;
                for (int g = 0; g < 10; ++g) {
                    const double xx = a0 + H * xg[g];
                    const double u = (xx - centre[d]) / sg;
                    sum += wg[g] * H * lag(P, a, xg[g]) * exp(-0.5 * u * u) / (sqrt(2.0 * M_PI) * sg);
                }
                I[d].push_back({{ci, a}, sum});
            }
        }
    }
    // z integrals over the screen
    const double lo = std::max(wl.z_bot, m.z0), hi = std::min(wl.z_top, m.z0 + m.Lz);
    double xq[3], wq[3];
    gauss01(3, xq, wq);
    for (int cz = 0; cz < m.nz; ++cz) {
        const double Hz = width_at(c, 2, cz);
        const double a0 = face_at(c, 2, cz), a1 = c->graded ? c->faces[2][cz + 1] : a0 + Hz;
        const double s0 = std::max(a0, lo), s1 = std::min(a1, hi);
        if (s1 <= s0) continue;
        for (int cc = 0; cc <= P; ++cc) {
            double Iz = 0;
            for (int g = 0; g < 3; ++g) Iz += wq[g] * (s1 - s0) * lag(P, cc, (s0 + (s1 - s0) * xq[g] - a0) / Hz);
            for (auto& ey : I[1])
                for (auto& ex : I[0]) {
                    const long long i = (long long)P * ex.first.first + ex.first.second;
                    const long long j = (long long)P * ey.first.first + ey.first.second;
                    const long long k = (long long)P * cz + cc;
                    out[i + (long long)c->grid.Nx * (j + (long long)c->grid.Ny * k)] += ex.second * ey.second * Iz;
                }
        }
    }
    return HT_OK;
}

// Rebuild Dirichlet values, static loads and source tables after changes.
// per-cell geometry of a graded mesh on the device: [4][nc] = volume, 1/hx,
// 1/hy, 1/hz (FP64 and FP32 copies)
int upload_geometry(ht_ctx* c) {
    if (!c->graded || !c->geo_dirty) return HT_OK;
    const Grid& g = c->grid;
    const size_t nc = (size_t)g.nc;
    std::vector<double> h(4 * nc);
    std::vector<float> f(4 * nc);
    for (int cz = 0; cz < g.ncz; ++cz)
        for (int cy = 0; cy < g.ncy; ++cy)
            for (int cx = 0; cx < g.ncx; ++cx) {
                const size_t id = cx + (size_t)g.ncx * (cy + (size_t)g.ncy * cz);
                const double hx = c->widths[0][cx], hy = c->widths[1][cy], hz = c->widths[2][cz];
                h[id] = hx * hy * hz;
                h[nc + id] = 1.0 / hx;
                h[2 * nc + id] = 1.0 / hy;
                h[3 * nc + id] = 1.0 / hz;
            }
    for (size_t i = 0; i < 4 * nc; ++i) f[i] = (float)h[i];
    if (!c->geo64 && cudaMalloc(&c->geo64, 4 * nc * sizeof(double)) != cudaSuccess)
        return fail(c, HT_ENOMEM, "graded-mesh geometry: allocation failed");
    if (!c->geo32 && cudaMalloc(&c->geo32, 4 * nc * sizeof(float)) != cudaSuccess)
        return fail(c, HT_ENOMEM, "graded-mesh geometry: allocation failed");
    HT_CUDA(c, cudaMemcpyAsync(c->geo64, h.data(), 4 * nc * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    HT_CUDA(c, cudaMemcpyAsync(c->geo32, f.data(), 4 * nc * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    HT_CUDA(c, cudaStreamSynchronize(c->stream));
    c->grid.geo64 = c->geo64;
    c->grid.geo32 = c->geo32;
    c->geo_dirty = false;
    return HT_OK;
}

int finalize_setup(ht_ctx* c) {
    if (!c->cells_set) return fail(c, HT_EINVAL, "ht_set_cells must be called before stepping");
    HT_TRY(upload_geometry(c));
    if (!c->bc_dirty && !c->loads_dirty) return HT_OK;
    const Grid& g = c->grid;
    const long long nn = g.nn;
    std::vector<double> gv(nn), Fs0(nn, 0.0), Fs1(nn, 0.0);
    for (int f = 0; f < 2; ++f) {
        std::fill(gv.begin(), gv.end(), 0.0);
        int mask = 0;
        std::vector<double>& Fs = f == 0 ? Fs0 : Fs1;
        for (int face = 0; face < 6; ++face) {
            const int axis = face / 2, side = face % 2;
            const int Nd[3] = {g.Nx, g.Ny, g.Nz};
            const int fixed = side ? Nd[axis] - 1 : 0;
            const int t1 = axis == 0 ? 1 : 0, t2 = axis == 2 ? 1 : 2;
            const int ncs[3] = {g.ncx, g.ncy, g.ncz};
            if (c->bc_type[f][face] == HT_BC_DIRICHLET) mask |= 1 << face;
            if (c->bc_type[f][face] == HT_BC_NONE) continue;
            const std::vector<double>& nodal = c->bc_nodal[f][face];
            auto face_node = [&](int a, int b) {
                int ijk[3];
                ijk[axis] = fixed;
                ijk[t1] = a;
                ijk[t2] = b;
                return ijk[0] + (long long)g.Nx * (ijk[1] + (long long)g.Ny * ijk[2]);
            };
            if (c->bc_type[f][face] == HT_BC_FLUX && !nodal.empty()) {
                // flux interpolated from its face-node values: F_i += sum_j M^face_ij q_j,
                // the face mass matrix a tensor product of 1D mass matrices per cell
                const int P = g.P;
                double M1[2][3][3];
                for (int c2 = 0; c2 < ncs[t2]; ++c2)
                    for (int c1 = 0; c1 < ncs[t1]; ++c1) {
                        for (int a = 0; a <= P; ++a)
                            for (int b = 0; b <= P; ++b) {
                                M1[0][a][b] = width_at(c, t1, c1) * phi_phi_int(P, a, b);
                                M1[1][a][b] = width_at(c, t2, c2) * phi_phi_int(P, a, b);
                            }
                        for (int b = 0; b <= P; ++b)
                            for (int a = 0; a <= P; ++a) {
                                double sum = 0.0;
                                for (int b2 = 0; b2 <= P; ++b2)
                                    for (int a2 = 0; a2 <= P; ++a2)
                                        sum += M1[0][a][a2] * M1[1][b][b2] *
                                               nodal[(P * c1 + a2) + (size_t)Nd[t1] * (P * c2 + b2)];
                                Fs[face_node(P * c1 + a, P * c2 + b)] += sum;
                            }
                    }
                continue;
            }
            for (int b = 0; b < Nd[t2]; ++b)
                for (int a = 0; a < Nd[t1]; ++a) {
                    const long long id = face_node(a, b);
                    if (c->bc_type[f][face] == HT_BC_DIRICHLET) {
                        gv[id] = nodal.empty() ? c->bc_val[f][face] : nodal[a + (size_t)Nd[t1] * b];
                    } else {
                        Fs[id] += c->bc_val[f][face] * node_int_axis(c, t1, a) * node_int_axis(c, t2, b);
                    }
                }
        }
        c->dmask[f] = mask;
        HT_CUDA(c, cudaMemcpyAsync(c->g[f], gv.data(), nn * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        HT_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    // pile surfaces at a prescribed temperature (heat Dirichlet rows)
    if (c->bc_dirty) HT_TRY(setup_pile_temperatures(c));
    // wells: head line source and (injection) lumped heat term
    std::map<long long, double> wd;
    for (const ht_well& w : c->wells) {
        std::map<long long, double> lw;
        HT_TRY(well_weights(c, w, lw));
        const double qlin = w.Q / (w.z_top - w.z_bot);
        for (auto& kv : lw) {
            Fs0[kv.first] += qlin * kv.second;
            // Dirichlet rows of the heat system stay identity rows
            if (w.Q > 0 && !node_on_dirichlet(c, HT_TEMP, kv.first)) {
                const double d = c->cw * qlin * kv.second;
                wd[kv.first] += d;
                Fs1[kv.first] += d * w.T_in;
            }
        }
    }
    HT_CUDA(c, cudaMemcpyAsync(c->Fstat[0], Fs0.data(), nn * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    HT_CUDA(c, cudaMemcpyAsync(c->Fstat[1], Fs1.data(), nn * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    // well diagonal list
    dfree(c->well_node);
    dfree(c->well_d);
    c->n_well_nodes = (int)wd.size();
    std::vector<int> wn;
    std::vector<double> wv;
    for (auto& kv : wd) { wn.push_back((int)kv.first); wv.push_back(kv.second); }
    if (!wn.empty()) {
        HT_TRY(dalloc(c, &c->well_node, wn.size()));
        HT_TRY(dalloc(c, &c->well_d, wv.size()));
        HT_CUDA(c, cudaMemcpyAsync(c->well_node, wn.data(), wn.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
        HT_CUDA(c, cudaMemcpyAsync(c->well_d, wv.data(), wv.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    }
    // the same coefficients as dense per-node arrays (zero off the wells)
    dfree(c->wdn64);
    dfree(c->wdn32);
    if (!wn.empty()) {
        std::vector<double> d64(nn, 0.0);
        std::vector<float> d32(nn, 0.0f);
        for (auto& kv : wd) { d64[kv.first] = kv.second; d32[kv.first] = (float)kv.second; }
        HT_TRY(dalloc(c, &c->wdn64, nn));
        HT_TRY(dalloc(c, &c->wdn32, nn));
        HT_CUDA(c, cudaMemcpyAsync(c->wdn64, d64.data(), nn * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        HT_CUDA(c, cudaMemcpyAsync(c->wdn32, d32.data(), nn * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        HT_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    // time-varying heat sources (piles, then boxes): CSR over unique nodes of
    // (source, weight); each source's time function q(t) = mean + amp sin(.)
    std::vector<ht_line_src> tf(c->piles);
    std::map<long long, std::vector<std::pair<int, double>>> pm;
    for (size_t s = 0; s < c->piles.size(); ++s) {
        const ht_line_src& p = c->piles[s];
        std::map<long long, double> lw;
        HT_TRY(line_weights(c, p.x, p.y, p.z_top, p.z_bot, lw, "line source"));
        for (auto& kv : lw) pm[kv.first].push_back({(int)s, kv.second});
    }
    for (const ht_box_src& b : c->boxes) {
        std::map<long long, double> bw;
        HT_TRY(box_weights(c, b, bw));
        const int s = (int)tf.size();
        ht_line_src f{};
        f.mean = b.mean;
        f.amp = b.amp;
        f.period = b.period;
        f.phase = b.phase;
        tf.push_back(f);
        for (auto& kv : bw) pm[kv.first].push_back({s, kv.second});
    }
    dfree(c->pile_node); dfree(c->pile_off); dfree(c->pile_src); dfree(c->pile_w); dfree(c->d_piles);
    c->n_pile_nodes = (int)pm.size();
    if (!pm.empty()) {
        std::vector<int> pn, po, ps;
        std::vector<double> pw;
        po.push_back(0);
        for (auto& kv : pm) {
            pn.push_back((int)kv.first);
            for (auto& e : kv.second) { ps.push_back(e.first); pw.push_back(e.second); }
            po.push_back((int)ps.size());
        }
        HT_TRY(dalloc(c, &c->pile_node, pn.size()));
        HT_TRY(dalloc(c, &c->pile_off, po.size()));
        HT_TRY(dalloc(c, &c->pile_src, ps.size()));
        HT_TRY(dalloc(c, &c->pile_w, pw.size()));
        HT_TRY(dalloc(c, &c->d_piles, tf.size()));
        HT_CUDA(c, cudaMemcpyAsync(c->pile_node, pn.data(), pn.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
        HT_CUDA(c, cudaMemcpyAsync(c->pile_off, po.data(), po.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
        HT_CUDA(c, cudaMemcpyAsync(c->pile_src, ps.data(), ps.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
        HT_CUDA(c, cudaMemcpyAsync(c->pile_w, pw.data(), pw.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        HT_CUDA(c, cudaMemcpyAsync(c->d_piles, tf.data(), tf.size() * sizeof(ht_line_src),
                                   cudaMemcpyHostToDevice, c->stream));
    }
    HT_CUDA(c, cudaStreamSynchronize(c->stream));
    c->bc_dirty = false;
    c->loads_dirty = false;
    return HT_OK;
}

int copy_in(ht_ctx* c, double* dst, const double* src, size_t n, int on_device) {
    HT_CUDA(c, cudaMemcpyAsync(dst, src, n * sizeof(double),
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    if (!on_device) HT_CUDA(c, cudaStreamSynchronize(c->stream));
    return HT_OK;
}

int copy_out(ht_ctx* c, double* dst, const double* src, size_t n, int on_device) {
    HT_CUDA(c, cudaMemcpyAsync(dst, src, n * sizeof(double),
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    HT_CUDA(c, cudaStreamSynchronize(c->stream));
    return HT_OK;
}

bool finite_pos(const double* a, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!(a[i] > 0.0) || !isfinite(a[i])) return false;
    return true;
}

int upload_cells(ht_ctx* c, double** d64, float** d32, const double* h, size_t nc) {
    if (!*d64) HT_TRY(dalloc(c, d64, nc));
    if (!*d32) HT_TRY(dalloc(c, d32, nc));
    std::vector<float> f(nc);
    for (size_t i = 0; i < nc; ++i) f[i] = (float)h[i];
    HT_CUDA(c, cudaMemcpyAsync(*d64, h, nc * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    HT_CUDA(c, cudaMemcpyAsync(*d32, f.data(), nc * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    HT_CUDA(c, cudaStreamSynchronize(c->stream));
    return HT_OK;
}

}  // namespace

int batch_prepare_diag(ht_ctx* c, double dt);

// Initial guess of one system of the step to t1, in c->x on entry (the field
// at t^n with its Dirichlet values): the extrapolation through the past
// fields replaces it when its residual under the FP32 operator is smaller.
// *used becomes 2 and *res that residual when it does; *res is the residual
// of the previous-step guess otherwise (-1 when no extrapolation was formed).
static int gate_extrapolated(ht_ctx* c, int field, double dt, double t1, int* used, double* res) {
    int deg = 0;
    HT_TRY(guess_extrapolate(c, field, t1, c->z, &deg));
    if (deg == 0) return HT_OK;
    double r0 = 0.0, r1 = 0.0;
    HT_TRY(fast_residual(c, field, dt, c->x, c->b, &r0));
    HT_TRY(fast_residual(c, field, dt, c->z, c->b, &r1));
    *res = r0;
    if (r1 < r0) {
        HT_CUDA(c, cudaMemcpyAsync(c->x, c->z, (size_t)c->grid.nn * sizeof(double), cudaMemcpyDeviceToDevice,
                                   c->stream));
        *used = 2;
        *res = r1;
    }
    c->guess_fast[field] = *res;   // the solve's first residual need not be formed in FP32 again
    return HT_OK;
}

// the learned guess against whatever c->x holds (ht_set_learned_guess)
static int gate_learned(ht_ctx* c, int field, double dt, int* used, double* res) {
    int won = 0;
    double r = -1.0;
    HT_TRY(learned_gate(c, field, dt, c->x, c->b, &won, &r));
    if (won) *used = 1;
    if (won || *res < 0) *res = r;
    if (r >= 0) c->guess_fast[field] = *res;
    return HT_OK;
}

// first part of a batched step: loads at t + dt, head right-hand side,
// initial iterate with Dirichlet values, diagonal
int batch_head_begin(ht_ctx* c, double dt) {
    // a batched step that ended early left the past fields half rotated
    if (c->guess_open) c->ghist = 0;
    c->guess_open = false;
    HT_TRY(finalize_setup(c));
    HT_TRY(launch_loads(c, c->t + dt));
    HT_TRY(launch_rhs(c, HT_HEAD, dt, c->h, c->b));
    HT_CUDA(c, cudaMemcpyAsync(c->x, c->h, (size_t)c->grid.nn * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    HT_TRY(set_dirichlet_values(c, HT_HEAD, c->x));
    if (c->opts.guess == HT_GUESS_EXTRAPOLATE) {
        c->guess_open = true;
        int used = 0;
        double res = -1.0;
        HT_TRY(gate_extrapolated(c, HT_HEAD, dt, c->t + dt, &used, &res));
    }
    return batch_prepare_diag(c, dt);
}

// last part of a batched step: store the head, then the heat solve with the
// Darcy flux of the new head (single-problem path)
int batch_head_end_and_heat(ht_ctx* c, double dt, ht_step_stats* st) {
    const size_t n = (size_t)c->grid.nn;
    HT_CUDA(c, cudaMemcpyAsync(c->h, c->x, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    HT_TRY(launch_darcy_qp(c, c->h));
    HT_TRY(launch_rhs(c, HT_TEMP, dt, c->T, c->b));
    HT_CUDA(c, cudaMemcpyAsync(c->x, c->T, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    HT_TRY(set_dirichlet_values(c, HT_TEMP, c->x));
    st->guess_res_heat = -1.0;
    if (c->guess_open) HT_TRY(gate_extrapolated(c, HT_TEMP, dt, c->t + dt, &st->guess_heat, &st->guess_res_heat));
    HT_TRY(solve_heat(c, dt, c->x, c->b, &st->iters_heat, &st->outer_heat, &st->res_heat));
    HT_CUDA(c, cudaMemcpyAsync(c->T, c->x, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    HT_CUDA(c, cudaStreamSynchronize(c->stream));
    if (c->guess_open) guess_commit(c, c->t);   // both systems recorded their fields at t^n
    c->guess_open = false;
    c->t += dt;
    st->t = c->t;
    return HT_OK;
}

int prof_flush(ht_ctx* c) {
    if (c->ev_used == 0) return HT_OK;
    HT_CUDA(c, cudaEventSynchronize(c->ev_pool[2 * c->ev_used - 1]));
    for (size_t i = 0; i < c->ev_used; ++i) {
        float ms = 0.f;
        HT_CUDA(c, cudaEventElapsedTime(&ms, c->ev_pool[2 * i], c->ev_pool[2 * i + 1]));
        c->prof_ms[c->ev_kind[i]].push_back(ms);
        c->prof_w[c->ev_kind[i]].push_back((float)c->ev_weight[i]);
    }
    c->ev_used = 0;
    c->ev_kind.clear();
    c->ev_weight.clear();
    return HT_OK;
}

int prof_begin(ht_ctx* c, int kind) {
    if (!c->prof_on) return HT_OK;
    if (c->ev_pool.empty()) {
        c->ev_pool.resize(4096);
        for (auto& e : c->ev_pool) HT_CUDA(c, cudaEventCreate(&e));
    }
    if (2 * c->ev_used + 2 > c->ev_pool.size()) HT_TRY(prof_flush(c));
    HT_CUDA(c, cudaEventRecord(c->ev_pool[2 * c->ev_used], c->stream));
    c->ev_kind.push_back(kind);
    c->ev_weight.push_back(1);
    return HT_OK;
}

int prof_end(ht_ctx* c) {
    if (!c->prof_on) return HT_OK;
    HT_CUDA(c, cudaEventRecord(c->ev_pool[2 * c->ev_used + 1], c->stream));
    c->ev_used += 1;
    return HT_OK;
}

int prof_end_weighted(ht_ctx* c, int weight) {
    if (!c->prof_on) return HT_OK;
    c->ev_weight.back() = weight;
    return prof_end(c);
}

void prof_drop_last(ht_ctx* c) {
    if (c->ev_used == 0 || c->ev_kind.empty()) return;
    c->ev_used -= 1;
    c->ev_kind.pop_back();
    c->ev_weight.pop_back();
}

}  // namespace ht

using namespace ht;

extern "C" {

int ht_default_solver(ht_solver_opts* o) {
    if (!o) return HT_EINVAL;
    memset(o, 0, sizeof(*o));
    o->tol = 1e-10;
    o->max_iter = 20000;
    o->krylov = HT_KRYLOV_GMRES;
    o->restart = 100;
    o->precond = HT_PREC_JACOBI;
    o->cheb_degree = 4;
    o->precision = HT_FP64;
    o->inner_tol = 1e-4;
    o->max_outer = 30;
    o->check_every = 8;
    o->use_graphs = 1;
    o->guess = HT_GUESS_EXTRAPOLATE;
    return HT_OK;
}

int ht_create(ht_ctx** out, const ht_mesh* mesh, int device, void* cuda_stream) {
    if (!out || !mesh) { g_create_error = "null argument"; return HT_EINVAL; }
    *out = nullptr;
    if (mesh->order != 1 && mesh->order != 2) { g_create_error = "order must be 1 or 2"; return HT_EINVAL; }
    if (mesh->nx < 1 || mesh->ny < 1 || mesh->nz < 1 || !(mesh->Lx > 0) || !(mesh->Ly > 0) || !(mesh->Lz > 0)) {
        g_create_error = "mesh sizes must be positive";
        return HT_EINVAL;
    }
    {
        // counts in doubles (no integer overflow): node indices and the largest
        // per-cell table index, 3 (P+1)^3 cells (Gauss-point velocities), must fit int
        const double Pd = mesh->order, nq = (Pd + 1) * (Pd + 1) * (Pd + 1);
        const double nnd = (Pd * mesh->nx + 1) * (Pd * mesh->ny + 1) * (Pd * mesh->nz + 1);
        const double ncd = (double)mesh->nx * mesh->ny * mesh->nz;
        if (nnd > 2.0e9 || 3.0 * nq * ncd > (double)INT_MAX) {
            g_create_error = "mesh too large for 32-bit node and cell tables";
            return HT_EINVAL;
        }
    }
    const long long P = mesh->order;
    const long long nn = (P * mesh->nx + 1) * (P * mesh->ny + 1) * (P * mesh->nz + 1);
    ht_ctx* c = new ht_ctx();
    c->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) {
        g_create_error = std::string("cudaSetDevice: ") + cudaGetErrorString(e);
        delete c;
        return HT_ECUDA;
    }
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            g_create_error = "cudaStreamCreate failed";
            delete c;
            return HT_ECUDA;
        }
        c->own_stream = true;
    }
    c->mesh = *mesh;
    Grid& g = c->grid;
    g.P = mesh->order;
    g.ncx = mesh->nx; g.ncy = mesh->ny; g.ncz = mesh->nz;
    g.Nx = g.P * g.ncx + 1; g.Ny = g.P * g.ncy + 1; g.Nz = g.P * g.ncz + 1;
    g.nn = nn;
    g.nc = (long long)mesh->nx * mesh->ny * mesh->nz;
    g.dmask = 0;
    c->H[0] = mesh->Lx / mesh->nx; c->H[1] = mesh->Ly / mesh->ny; c->H[2] = mesh->Lz / mesh->nz;
    build_elem(c);
    ht_default_solver(&c->opts);
    const size_t N = (size_t)nn, NC = (size_t)g.nc;
    const size_t NQ = (size_t)(g.P + 1) * (g.P + 1) * (g.P + 1);
    int rc = HT_OK;
    double** v64[] = {&c->h, &c->T, &c->g[0], &c->g[1], &c->Fstat[0], &c->Fstat[1], &c->F[0], &c->F[1],
                      &c->extra[0], &c->extra[1], &c->x, &c->r, &c->z, &c->p, &c->q, &c->b, &c->D,
                      &c->rh, &c->v, &c->s, &c->tv, &c->ph, &c->sh, &c->z2};
    for (double** pp : v64)
        if (rc == HT_OK) rc = dalloc(c, pp, N);
    float** v32[] = {&c->x32, &c->r32, &c->z32, &c->p32, &c->q32, &c->D32, &c->rh32, &c->v32,
                     &c->s32, &c->t32, &c->ph32, &c->sh32, &c->zz32, &c->d32, &c->h32};
    for (float** pp : v32)
        if (rc == HT_OK) rc = dalloc(c, pp, N);
    if (rc == HT_OK) rc = dalloc(c, &c->qs64, 3 * NQ * NC);
    if (rc == HT_OK) rc = dalloc(c, &c->qs32, 3 * NQ * NC);
    // element buffers of the two-pass kernels behind kElemPad zeros: node
    // gathers read E[-1] for absent neighbour cells, element passes write
    // only E[0 .. NQ * NC)
    if (rc == HT_OK) rc = dalloc(c, &c->E32, NQ * NC + kElemPad);
    if (rc == HT_OK) rc = dalloc(c, &c->E64, NQ * NC + kElemPad);
    if (rc == HT_OK && cudaMemsetAsync(c->E32, 0, (NQ * NC + kElemPad) * sizeof(float), c->stream) != cudaSuccess) rc = HT_ECUDA;
    if (rc == HT_OK && cudaMemsetAsync(c->E64, 0, (NQ * NC + kElemPad) * sizeof(double), c->stream) != cudaSuccess) rc = HT_ECUDA;
    const int G = vec_grid(c), tiles = apply_tiles(c);
    // the two-pass node gather writes one partial per 128-node run of a layer and
    // layer split, at most one wave of 128-thread CTAs (16 per SM) beyond one split
    const int node_blocks = ((g.Nx + 31) / 32) * ((g.Ny + 3) / 4) + 16 * std::max(c->num_sms, 148);
    c->part_stride = std::max(std::max(G, tiles), node_blocks) + 32;
    if (rc == HT_OK) rc = dalloc(c, &c->part, (size_t)(kMaxRestart + 8) * c->part_stride);
    if (rc == HT_OK) rc = dalloc(c, &c->gm, 2);
    if (rc == HT_OK) rc = dalloc(c, &c->scal, 4);
    if (rc == HT_OK && cudaMallocHost(&c->scal_host, 4 * sizeof(Scal)) != cudaSuccess) rc = HT_ENOMEM;
    if (rc == HT_OK) {
        for (double* p : {c->h, c->T, c->extra[0], c->extra[1], c->Fstat[0], c->Fstat[1], c->g[0], c->g[1]})
            if (cudaMemsetAsync(p, 0, N * sizeof(double), c->stream) != cudaSuccess) rc = HT_ECUDA;
        if (cudaMemsetAsync(c->qs64, 0, 3 * NQ * NC * sizeof(double), c->stream) != cudaSuccess) rc = HT_ECUDA;
        if (cudaMemsetAsync(c->qs32, 0, 3 * NQ * NC * sizeof(float), c->stream) != cudaSuccess) rc = HT_ECUDA;
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) rc = HT_ECUDA;
    }
    if (rc != HT_OK) {
        g_create_error = c->err.empty() ? "allocation failed" : c->err;
        ht_destroy(c);
        return rc;
    }
    *out = c;
    return HT_OK;
}

void ht_destroy(ht_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (auto* gr : {&c->g_cg[0], &c->g_cg[1], &c->g_bi[0], &c->g_bi[1], &c->g_cg1, &c->g_bi1})
        if (gr->exec) cudaGraphExecDestroy(gr->exec);
    double** v64[] = {&c->h, &c->T, &c->g[0], &c->g[1], &c->Fstat[0], &c->Fstat[1], &c->F[0], &c->F[1],
                      &c->extra[0], &c->extra[1], &c->x, &c->r, &c->z, &c->p, &c->q, &c->b, &c->D,
                      &c->rh, &c->v, &c->s, &c->tv, &c->ph, &c->sh, &c->z2, &c->K64, &c->lam64,
                      &c->cT64, &c->qs64, &c->part, &c->pile_w, &c->well_d, &c->E64, &c->wdn64};
    for (double** pp : v64) dfree(*pp);
    float** v32[] = {&c->x32, &c->r32, &c->z32, &c->p32, &c->q32, &c->D32, &c->rh32, &c->v32, &c->s32,
                     &c->t32, &c->ph32, &c->sh32, &c->zz32, &c->d32, &c->K32, &c->lam32, &c->cT32, &c->qs32,
                     &c->E32, &c->wdn32, &c->h32};
    for (float** pp : v32) dfree(*pp);
    dfree(c->pile_node); dfree(c->pile_off); dfree(c->pile_src); dfree(c->d_piles); dfree(c->well_node);
    dfree(c->ptemp_node); dfree(c->ptemp_pile); dfree(c->d_ptemp); dfree(c->dint);
    dfree(c->dint_a64); dfree(c->dint_b64); dfree(c->dint_a32);
    dfree(c->xdf); dfree(c->hdf); dfree(c->geo64); dfree(c->geo32);
    dfree(c->scal);
    dfree(c->gm);
    dfree(c->V64);
    dfree(c->V32);
    if (c->scal_host) cudaFreeHost(c->scal_host);
    for (auto& e : c->ev_pool) cudaEventDestroy(e);
    learned_free(c);
    guess_free(c);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

const char* ht_last_error(const ht_ctx* c) {
    if (!c) return g_create_error.c_str();
    return c->err.c_str();
}

int ht_sizes(const ht_ctx* c, size_t* n_nodes, size_t* n_cells) {
    if (!c) return HT_EINVAL;
    if (n_nodes) *n_nodes = (size_t)c->grid.nn;
    if (n_cells) *n_cells = (size_t)c->grid.nc;
    return HT_OK;
}

int ht_set_cells(ht_ctx* c, const double* K, const double* lambda, const double* cT, double lambda_u,
                 double cT_u, double cw, double Ss) {
    if (!c || !K) return HT_EINVAL;
    cudaSetDevice(c->device);
    const size_t nc = (size_t)c->grid.nc;
    if (!finite_pos(K, nc)) return fail(c, HT_EINVAL, "K must be positive and finite in every cell");
    if (lambda && !finite_pos(lambda, nc)) return fail(c, HT_EINVAL, "lambda must be positive and finite");
    if (cT && !finite_pos(cT, nc)) return fail(c, HT_EINVAL, "cT must be positive and finite");
    if ((!lambda && !(lambda_u > 0)) || (!cT && !(cT_u > 0)) || !(cw >= 0) || !(Ss > 0) || !isfinite(cw) ||
        !isfinite(Ss) || !isfinite(lambda_u) || !isfinite(cT_u))
        return fail(c, HT_EINVAL, "uniform coefficients must be positive and finite");
    HT_TRY(upload_cells(c, &c->K64, &c->K32, K, nc));
    if (lambda) HT_TRY(upload_cells(c, &c->lam64, &c->lam32, lambda, nc));
    else { dfree(c->lam64); dfree(c->lam32); }
    if (cT) HT_TRY(upload_cells(c, &c->cT64, &c->cT32, cT, nc));
    else { dfree(c->cT64); dfree(c->cT32); }
    c->lam_u = lambda_u;
    c->cT_u = cT_u;
    c->cw = cw;
    c->Ss = Ss;
    c->cells_set = true;
    c->loads_dirty = true;   // well heat terms depend on c_w
    c->cheb_dt[0] = c->cheb_dt[1] = -1.0;   // operator changed: re-estimate the spectrum
    return HT_OK;
}

int ht_set_bc(ht_ctx* c, int field, int face, int type, double value) {
    if (!c) return HT_EINVAL;
    if (field != HT_HEAD && field != HT_TEMP) return fail(c, HT_EINVAL, "field must be HT_HEAD or HT_TEMP");
    if (face < 0 || face > 5) return fail(c, HT_EINVAL, "face must be 0..5");
    if (type < HT_BC_NONE || type > HT_BC_FLUX) return fail(c, HT_EINVAL, "unknown boundary type %d", type);
    if (!isfinite(value)) return fail(c, HT_EINVAL, "boundary value must be finite");
    c->bc_type[field][face] = type;
    c->bc_val[field][face] = value;
    c->bc_nodal[field][face].clear();
    c->seasonal[field][face].on = 0;
    c->bc_dirty = true;
    c->cheb_dt[field] = -1.0;
    return HT_OK;
}

int ht_set_spacing(ht_ctx* c, int axis, const double* widths, int n) {
    if (!c) return HT_EINVAL;
    if (axis < 0 || axis > 2) return fail(c, HT_EINVAL, "axis must be 0, 1 or 2");
    if (!widths || n != axis_cells(c, axis))
        return fail(c, HT_EINVAL, "axis %d has %d cells, got %d widths", axis, axis_cells(c, axis), n);
    for (int k = 0; k < n; ++k)
        if (!(widths[k] > 0) || !isfinite(widths[k])) return fail(c, HT_EINVAL, "width %d must be positive", k);
    if (!c->graded) {   // the other axes keep their uniform widths
        for (int d = 0; d < 3; ++d) {
            const int nd = axis_cells(c, d);
            c->widths[d].assign(nd, c->H[d]);
        }
    }
    c->widths[axis].assign(widths, widths + n);
    for (int d = 0; d < 3; ++d) {
        const int nd = axis_cells(c, d);
        c->faces[d].resize(nd + 1);
        const double org = axis_origin(c, d);
        double cum = 0.0;
        for (int k = 0; k <= nd; ++k) {
            c->faces[d][k] = org + cum;
            if (k < nd) cum += c->widths[d][k];
        }
        if (d == 0) c->mesh.Lx = cum;
        if (d == 1) c->mesh.Ly = cum;
        if (d == 2) c->mesh.Lz = cum;
        c->H[d] = cum / nd;   // mean width (nominal cell size)
    }
    for (auto* gr : {&c->g_cg[0], &c->g_cg[1], &c->g_bi[0], &c->g_bi[1], &c->g_cg1, &c->g_bi1})
        gr->dt = -1.0;   // captured launches hold the element constants: recapture
    c->graded = true;
    c->geo_dirty = true;
    c->bc_dirty = true;
    c->loads_dirty = true;
    c->cheb_dt[0] = c->cheb_dt[1] = -1.0;
    build_elem(c);
    return HT_OK;
}

int ht_set_seasonal_face(ht_ctx* c, int field, int face, double mean, double amp, double period, double phase) {
    if (!c) return HT_EINVAL;
    if (field != HT_HEAD && field != HT_TEMP) return fail(c, HT_EINVAL, "field must be HT_HEAD or HT_TEMP");
    if (face < 0 || face > 5) return fail(c, HT_EINVAL, "face must be 0..5");
    if (!isfinite(mean) || !isfinite(amp) || !isfinite(phase) || !(period > 0) || !isfinite(period))
        return fail(c, HT_EINVAL, "seasonal face needs finite mean, amplitude and phase and a positive period");
    c->bc_type[field][face] = HT_BC_DIRICHLET;
    c->bc_val[field][face] = mean;
    c->bc_nodal[field][face].clear();
    c->seasonal[field][face] = ht_ctx::Seasonal{1, mean, amp, period, phase};
    c->bc_dirty = true;
    c->cheb_dt[field] = -1.0;
    return HT_OK;
}

int ht_set_pile_temperatures(ht_ctx* c, int n, const double* rows) {
    if (!c || n < 0 || (n > 0 && !rows)) return HT_EINVAL;
    for (int p = 0; p < n; ++p) {
        const double* r = rows + 9 * (size_t)p;
        for (int q = 0; q < 9; ++q)
            if (!isfinite(r[q])) return fail(c, HT_EINVAL, "pile temperature row %d has a non-finite entry", p);
        if (r[4] < 0 || !(r[7] > 0))
            return fail(c, HT_EINVAL, "pile temperature row %d: radius >= 0 and period > 0 are required", p);
        const ht_mesh& m = c->mesh;
        if (std::max(r[2], r[3]) < m.z0 || std::min(r[2], r[3]) > m.z0 + m.Lz)
            return fail(c, HT_EINVAL, "pile temperature row %d lies outside the mesh in z", p);
    }
    c->ptemp_rows.assign(rows, rows + 9 * (size_t)n);
    c->bc_dirty = true;
    return HT_OK;
}

int ht_face_nodes(const ht_ctx* c, int face, size_t* n) {
    if (!c || !n || face < 0 || face > 5) return HT_EINVAL;
    const Grid& g = c->grid;
    const size_t Nd[3] = {(size_t)g.Nx, (size_t)g.Ny, (size_t)g.Nz};
    const int axis = face / 2;
    *n = Nd[axis == 0 ? 1 : 0] * Nd[axis == 2 ? 1 : 2];
    return HT_OK;
}

int ht_set_bc_values(ht_ctx* c, int field, int face, int type, const double* values, size_t n) {
    if (!c) return HT_EINVAL;
    if (field != HT_HEAD && field != HT_TEMP) return fail(c, HT_EINVAL, "field must be HT_HEAD or HT_TEMP");
    if (face < 0 || face > 5) return fail(c, HT_EINVAL, "face must be 0..5");
    if (type != HT_BC_DIRICHLET && type != HT_BC_FLUX)
        return fail(c, HT_EINVAL, "per-node values need HT_BC_DIRICHLET or HT_BC_FLUX, got %d", type);
    size_t nf = 0;
    ht_face_nodes(c, face, &nf);
    if (!values || n != nf) return fail(c, HT_EINVAL, "face %d has %zu nodes, got %zu values", face, nf, n);
    for (size_t i = 0; i < n; ++i)
        if (!isfinite(values[i])) return fail(c, HT_EINVAL, "boundary value %zu is not finite", i);
    c->bc_type[field][face] = type;
    c->bc_val[field][face] = 0.0;
    c->bc_nodal[field][face].assign(values, values + n);
    c->bc_dirty = true;
    c->cheb_dt[field] = -1.0;
    return HT_OK;
}

int ht_set_state(ht_ctx* c, const double* h, const double* T, double t, int on_device) {
    if (!c) return HT_EINVAL;
    if (!isfinite(t)) return fail(c, HT_EINVAL, "time must be finite");
    cudaSetDevice(c->device);
    const size_t n = (size_t)c->grid.nn;
    if (h) HT_TRY(copy_in(c, c->h, h, n, on_device));
    if (T) HT_TRY(copy_in(c, c->T, T, n, on_device));
    c->t = t;
    c->ghist = 0;   // the extrapolated guess starts afresh from the new state
    c->guess_open = false;
    return HT_OK;
}

int ht_add_line_sources(ht_ctx* c, int n, const ht_line_src* src) {
    if (!c || n < 0 || (n > 0 && !src)) return HT_EINVAL;
    for (int i = 0; i < n; ++i) {
        const ht_line_src& s = src[i];
        if (!(s.z_top > s.z_bot) || !isfinite(s.mean) || !isfinite(s.amp) || !(s.period > 0) || !isfinite(s.phase))
            return fail(c, HT_EINVAL, "line source %d: invalid parameters", i);
        std::map<long long, double> probe;
        HT_TRY(line_weights(c, s.x, s.y, s.z_top, s.z_bot, probe, "line source"));
    }
    c->piles.insert(c->piles.end(), src, src + n);
    c->loads_dirty = true;
    return HT_OK;
}

int ht_add_box_sources(ht_ctx* c, int n, const ht_box_src* b) {
    if (!c || n < 0 || (n > 0 && !b)) return HT_EINVAL;
    const ht_mesh& m = c->mesh;
    const double eps = 1e-9 * std::max(m.Lx, std::max(m.Ly, m.Lz));
    for (int i = 0; i < n; ++i) {
        const ht_box_src& s = b[i];
        const double v[9] = {s.x0, s.x1, s.y0, s.y1, s.z, s.mean, s.amp, s.period, s.phase};
        for (double e : v)
            if (!isfinite(e)) return fail(c, HT_EINVAL, "box source %d: non-finite parameter", i);
        if (!(s.x1 > s.x0) || !(s.y1 > s.y0) || !(s.period > 0))
            return fail(c, HT_EINVAL, "box source %d: needs x1 > x0, y1 > y0 and period > 0", i);
        if (!(s.z >= m.z0 - eps && s.z <= m.z0 + m.Lz + eps))
            return fail(c, HT_EINVAL, "box source %d: plane z = %g lies outside the box", i, s.z);
        std::map<long long, double> probe;
        HT_TRY(box_weights(c, s, probe));
    }
    c->boxes.insert(c->boxes.end(), b, b + n);
    c->loads_dirty = true;
    return HT_OK;
}

int ht_add_wells(ht_ctx* c, int n, const ht_well* w) {
    if (!c || n < 0 || (n > 0 && !w)) return HT_EINVAL;
    for (int i = 0; i < n; ++i) {
        if (!isfinite(w[i].Q) || !isfinite(w[i].T_in) || !(w[i].sigma >= 0) || !isfinite(w[i].sigma))
            return fail(c, HT_EINVAL, "well %d: invalid parameters", i);
        std::map<long long, double> probe;
        HT_TRY(line_weights(c, w[i].x, w[i].y, w[i].z_top, w[i].z_bot, probe, "well"));
    }
    c->wells.insert(c->wells.end(), w, w + n);
    c->loads_dirty = true;
    return HT_OK;
}

int ht_set_extra_rhs(ht_ctx* c, int field, const double* F, int on_device) {
    if (!c) return HT_EINVAL;
    if (field != HT_HEAD && field != HT_TEMP) return fail(c, HT_EINVAL, "field must be HT_HEAD or HT_TEMP");
    cudaSetDevice(c->device);
    const size_t n = (size_t)c->grid.nn;
    if (!F) {
        HT_CUDA(c, cudaMemsetAsync(c->extra[field], 0, n * sizeof(double), c->stream));
        return HT_OK;
    }
    return copy_in(c, c->extra[field], F, n, on_device);
}

int ht_set_solver(ht_ctx* c, const ht_solver_opts* o) {
    if (!c || !o) return HT_EINVAL;
    if (!(o->tol > 0) || o->max_iter < 1) return fail(c, HT_EINVAL, "tol > 0 and max_iter >= 1 required");
    if (o->precision != HT_FP64 && o->precision != HT_MIXED) return fail(c, HT_EINVAL, "unknown precision");
    if (o->krylov != HT_KRYLOV_BICGSTAB && o->krylov != HT_KRYLOV_GMRES)
        return fail(c, HT_EINVAL, "unsupported Krylov method %d", o->krylov);
    if (o->krylov == HT_KRYLOV_GMRES && (o->restart < 2 || o->restart > ht::kMaxRestart))
        return fail(c, HT_EINVAL, "GMRES restart must be 2..%d", ht::kMaxRestart);
    if (o->precond != HT_PREC_JACOBI && o->precond != HT_PREC_CHEBYSHEV)
        return fail(c, HT_EINVAL, "unknown preconditioner");
    if (o->precond == HT_PREC_CHEBYSHEV && (o->cheb_degree < 1 || o->cheb_degree > 32))
        return fail(c, HT_EINVAL, "cheb_degree must be 1..32");
    if (o->z_chunks < 0) return fail(c, HT_EINVAL, "z_chunks must be >= 0");
    if (!(o->inner_tol >= 0 && o->inner_tol < 1) || !(o->inner_tol_heat >= 0 && o->inner_tol_heat < 1))
        return fail(c, HT_EINVAL, "inner tolerances must be in [0, 1)");
    if (o->apply_variant < HT_APPLY_AUTO || o->apply_variant > HT_APPLY_SINGLE_PASS)
        return fail(c, HT_EINVAL, "unknown apply variant %d", o->apply_variant);
    if (o->guess != HT_GUESS_PREVIOUS && o->guess != HT_GUESS_EXTRAPOLATE)
        return fail(c, HT_EINVAL, "unknown initial guess %d", o->guess);
    if (o->guess != HT_GUESS_EXTRAPOLATE) c->ghist = 0;   // past fields are kept only while extrapolating
    c->opts = *o;
    return HT_OK;
}


int ht_step(ht_ctx* c, double dt, ht_step_stats* st) {
    if (!c) return HT_EINVAL;
    if (!(dt > 0) || !isfinite(dt)) return fail(c, HT_EINVAL, "dt must be positive");
    cudaSetDevice(c->device);
    HT_TRY(finalize_setup(c));
    cudaEvent_t ev[4];
    for (auto& e : ev) HT_CUDA(c, cudaEventCreate(&e));
    const size_t n = (size_t)c->grid.nn;
    const double t1 = c->t + dt;
    ht_step_stats s{};
    int rc = HT_OK;
    cudaEventRecord(ev[0], c->stream);
    rc = launch_loads(c, t1);
    if (rc == HT_OK) rc = learned_begin(c);     // features include the heat loads at t^{n+1}
    cudaEventRecord(ev[1], c->stream);
    // head: b = S_s M h^n + dt F_h lifted; x0 = h^n with Dirichlet values
    if (rc == HT_OK) rc = launch_rhs(c, HT_HEAD, dt, c->h, c->b);
    if (rc == HT_OK && cudaMemcpyAsync(c->x, c->h, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
        rc = fail(c, HT_ECUDA, "copy failed");
    if (rc == HT_OK) rc = set_dirichlet_values(c, HT_HEAD, c->x);
    s.guess_res_head = s.guess_res_heat = -1.0;
    if (c->guess_open) c->ghist = 0;   // a batched step that ended early
    c->guess_open = false;
    const bool extrap = c->opts.guess == HT_GUESS_EXTRAPOLATE;
    if (rc == HT_OK && extrap) rc = gate_extrapolated(c, HT_HEAD, dt, t1, &s.guess_head, &s.guess_res_head);
    if (rc == HT_OK) rc = gate_learned(c, HT_HEAD, dt, &s.guess_head, &s.guess_res_head);
    if (rc == HT_OK) rc = solve_head(c, dt, c->x, c->b, &s.iters_head, &s.outer_head, &s.res_head);
    int rc_head = rc;
    if (rc == HT_OK || rc == HT_ENOCONV)
        if (cudaMemcpyAsync(c->h, c->x, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
            rc = fail(c, HT_ECUDA, "copy failed");
    cudaEventRecord(ev[2], c->stream);
    if (rc == HT_OK) {
        // heat with q = -K grad h^{n+1}
        rc = launch_darcy_qp(c, c->h);
        if (rc == HT_OK) rc = launch_rhs(c, HT_TEMP, dt, c->T, c->b);
        if (rc == HT_OK && cudaMemcpyAsync(c->x, c->T, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
            rc = fail(c, HT_ECUDA, "copy failed");
        if (rc == HT_OK) rc = set_dirichlet_values(c, HT_TEMP, c->x);
        if (rc == HT_OK && extrap) rc = gate_extrapolated(c, HT_TEMP, dt, t1, &s.guess_heat, &s.guess_res_heat);
        if (rc == HT_OK) rc = gate_learned(c, HT_TEMP, dt, &s.guess_heat, &s.guess_res_heat);
        if (rc == HT_OK) rc = solve_heat(c, dt, c->x, c->b, &s.iters_heat, &s.outer_heat, &s.res_heat);
        if (rc == HT_OK || rc == HT_ENOCONV)
            if (cudaMemcpyAsync(c->T, c->x, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
                rc = fail(c, HT_ECUDA, "copy failed");
    }
    if (rc == HT_OK) {
        // the step is complete: history for the learned guess (state update below)
        const double t_save = c->t;
        (void)t_save;
        rc = learned_end(c);
    }
    cudaEventRecord(ev[3], c->stream);
    cudaEventSynchronize(ev[3]);
    float ms;
    cudaEventElapsedTime(&ms, ev[0], ev[1]); s.ms_loads = ms;
    cudaEventElapsedTime(&ms, ev[1], ev[2]); s.ms_head = ms;
    cudaEventElapsedTime(&ms, ev[2], ev[3]); s.ms_heat = ms;
    cudaEventElapsedTime(&ms, ev[0], ev[3]); s.ms_total = ms;
    for (auto& e : ev) cudaEventDestroy(e);
    // the past fields of the extrapolated guess: both systems recorded their
    // state at t^n; a step that failed anywhere forgets them
    if (extrap) {
        if (rc == HT_OK) guess_commit(c, c->t);
        else c->ghist = 0;
    }
    if (rc == HT_OK || rc == HT_ENOCONV) c->t = t1;
    s.t = c->t;
    s.status = rc;
    if (st) *st = s;
    (void)rc_head;
    return rc;
}

int ht_get_field(ht_ctx* c, int field, double* dst, size_t n, int on_device) {
    if (!c || !dst) return HT_EINVAL;
    cudaSetDevice(c->device);
    if (field == HT_HEAD || field == HT_TEMP) {
        if (n != (size_t)c->grid.nn) return fail(c, HT_EINVAL, "size %zu != node count %lld", n, c->grid.nn);
        return copy_out(c, dst, field == HT_HEAD ? c->h : c->T, n, on_device);
    }
    if (field >= HT_QX && field <= HT_QZ) {
        if (n != (size_t)c->grid.nc) return fail(c, HT_EINVAL, "size %zu != cell count %lld", n, c->grid.nc);
        if (!c->cells_set) return fail(c, HT_EINVAL, "cells not set");
        HT_TRY(launch_cell_flux(c, c->h, field - HT_QX, c->z));
        return copy_out(c, dst, c->z, n, on_device);
    }
    return fail(c, HT_EINVAL, "unknown field %d", field);
}

int ht_get_time(const ht_ctx* c, double* t) {
    if (!c || !t) return HT_EINVAL;
    *t = c->t;
    return HT_OK;
}

int ht_apply(ht_ctx* c, int field, double dt, const double* x, double* y, int on_device) {
    if (!c || !x || !y) return HT_EINVAL;
    if (field != HT_HEAD && field != HT_TEMP) return fail(c, HT_EINVAL, "field must be HT_HEAD or HT_TEMP");
    if (!(dt > 0)) return fail(c, HT_EINVAL, "dt must be positive");
    cudaSetDevice(c->device);
    HT_TRY(finalize_setup(c));
    const size_t n = (size_t)c->grid.nn;
    HT_TRY(copy_in(c, c->z, x, n, on_device));
    if (field == HT_TEMP) HT_TRY(launch_darcy_qp(c, c->h));
    HT_TRY(launch_apply64(c, field, dt, c->z, c->q, nullptr, nullptr, nullptr));
    return copy_out(c, y, c->q, n, on_device);
}

int ht_diag(ht_ctx* c, int field, double dt, double* d, int on_device) {
    if (!c || !d) return HT_EINVAL;
    if (field != HT_HEAD && field != HT_TEMP) return fail(c, HT_EINVAL, "field must be HT_HEAD or HT_TEMP");
    cudaSetDevice(c->device);
    HT_TRY(finalize_setup(c));
    if (field == HT_TEMP) HT_TRY(launch_darcy_qp(c, c->h));
    HT_TRY(launch_diag(c, field, dt, c->q));
    return copy_out(c, d, c->q, (size_t)c->grid.nn, on_device);
}

int ht_residual(ht_ctx* c, int field, double dt, const double* x, const double* b, int emulated, int on_device,
                double* rel) {
    if (!c || !x || !b || !rel) return HT_EINVAL;
    if (field != HT_HEAD && field != HT_TEMP) return fail(c, HT_EINVAL, "field must be HT_HEAD or HT_TEMP");
    if (!(dt > 0)) return fail(c, HT_EINVAL, "dt must be positive");
    cudaSetDevice(c->device);
    HT_TRY(finalize_setup(c));
    const size_t n = (size_t)c->grid.nn;
    HT_TRY(copy_in(c, c->z, x, n, on_device));
    HT_TRY(copy_in(c, c->v, b, n, on_device));
    if (field == HT_TEMP) HT_TRY(launch_darcy_qp(c, c->h));
    int np = 0;
    if (emulated && !(field == HT_TEMP && !heat_fused_ok(c))) {
        HT_TRY(launch_resid_df(c, field, dt, c->z, c->v, c->r32, c->part, &np));
    } else {
        HT_TRY(launch_apply64(c, field, dt, c->z, c->q, nullptr, nullptr, nullptr));
        HT_TRY(launch_resid64(c, c->v, c->q, c->part, &np));
    }
    HT_TRY(launch_norms(c, np, 3));
    HT_CUDA(c, cudaMemcpyAsync(c->scal_host + 3, c->scal + 3, sizeof(ht::Scal), cudaMemcpyDeviceToHost, c->stream));
    HT_CUDA(c, cudaStreamSynchronize(c->stream));
    const ht::Scal s = c->scal_host[3];
    *rel = s.bb > 0 ? sqrt(s.rr / s.bb) : sqrt(s.rr);
    return HT_OK;
}

int ht_rhs(ht_ctx* c, int field, double dt, double* b, int on_device) {
    if (!c || !b) return HT_EINVAL;
    if (field != HT_HEAD && field != HT_TEMP) return fail(c, HT_EINVAL, "field must be HT_HEAD or HT_TEMP");
    cudaSetDevice(c->device);
    HT_TRY(finalize_setup(c));
    HT_TRY(launch_loads(c, c->t + dt));
    if (field == HT_TEMP) HT_TRY(launch_darcy_qp(c, c->h));
    HT_TRY(launch_rhs(c, field, dt, field == HT_HEAD ? c->h : c->T, c->q));
    return copy_out(c, b, c->q, (size_t)c->grid.nn, on_device);
}

int ht_profile(ht_ctx* c, int on) {
    if (!c) return HT_EINVAL;
    cudaSetDevice(c->device);
    HT_TRY(prof_flush(c));
    c->prof_on = on;
    c->n_launch = 0;
    for (auto& v : c->prof_ms) v.clear();
    for (auto& v : c->prof_w) v.clear();
    return HT_OK;
}

int ht_profile_read(ht_ctx* c, ht_profile_stats* out) {
    if (!c || !out) return HT_EINVAL;
    cudaSetDevice(c->device);
    HT_TRY(prof_flush(c));
    memset(out, 0, sizeof(*out));
    out->launches = c->n_launch;
    long long* cnt[HT_PROF_KINDS] = {&out->head_applies, &out->heat_applies, &out->head_applies_fp32,
                                  &out->heat_applies_fp32, &out->cg_iters, &out->bicgstab_iters};
    double* ms[HT_PROF_KINDS] = {&out->head_apply_ms, &out->heat_apply_ms, &out->head_apply_ms_fp32,
                              &out->heat_apply_ms_fp32, &out->cg_iter_ms, &out->bicgstab_iter_ms};
    for (int k = 0; k < HT_PROF_KINDS; ++k) {
        std::vector<float> v = c->prof_ms[k];
        if (v.empty()) continue;
        if (k == HT_PROF_CG_ITER || k == HT_PROF_BICGSTAB_ITER) {
            // timed check intervals in which every iteration did work
            for (size_t i = 0; i < v.size(); ++i) {
                *cnt[k] += (long long)c->prof_w[k][i];
                *ms[k] += v[i];
            }
            continue;
        }
        std::vector<float> srt = v;
        std::nth_element(srt.begin(), srt.begin() + srt.size() / 2, srt.end());
        const float med = srt[srt.size() / 2];
        // launches that returned at once (solve already converged) take a tiny
        // fraction of a working launch; leave them out of the average
        for (float x : v)
            if (x >= 0.25f * med) { *cnt[k] += 1; *ms[k] += x; }
    }
    return HT_OK;
}

int ht_head_apply_dot_noalloc(const ht_mesh* mesh, int dirichlet_faces, double Ss, double dt, const double* K,
                              const double* x, double* y, double* xAx, int device, void* cuda_stream, char* msg,
                              size_t msg_len) {
    if (msg && msg_len) msg[0] = 0;
    if (!mesh || !K || !x || !y || !xAx) {
        if (msg && msg_len) snprintf(msg, msg_len, "null argument");
        return HT_EINVAL;
    }
    if ((mesh->order != 1 && mesh->order != 2) || mesh->nx < 1 || mesh->ny < 1 || mesh->nz < 1 ||
        !(mesh->Lx > 0) || !(mesh->Ly > 0) || !(mesh->Lz > 0) || !(Ss > 0) || !(dt > 0) ||
        dirichlet_faces < 0 || dirichlet_faces > 63) {
        if (msg && msg_len) snprintf(msg, msg_len, "invalid mesh, coefficient or face mask");
        return HT_EINVAL;
    }
    {
        // node and cell counts without integer overflow (doubles are exact far
        // beyond the limit); the kernels index nodes and cells with int
        const double P = mesh->order;
        const double nn = (P * mesh->nx + 1) * (P * mesh->ny + 1) * (P * mesh->nz + 1);
        const double nc = (double)mesh->nx * mesh->ny * mesh->nz;
        if (nn > (double)INT_MAX || nc > (double)INT_MAX) {
            if (msg && msg_len) snprintf(msg, msg_len, "mesh too large: %.0f nodes, %.0f cells", nn, nc);
            return HT_EINVAL;
        }
    }
    Grid g{};
    g.P = mesh->order;
    g.ncx = mesh->nx; g.ncy = mesh->ny; g.ncz = mesh->nz;
    g.Nx = g.P * g.ncx + 1; g.Ny = g.P * g.ncy + 1; g.Nz = g.P * g.ncz + 1;
    g.nn = (long long)g.Nx * g.Ny * g.Nz;
    g.nc = (long long)g.ncx * g.ncy * g.ncz;
    g.dmask = dirichlet_faces;
    // reference-element constants on the stack (no allocation)
    const double H[3] = {mesh->Lx / mesh->nx, mesh->Ly / mesh->ny, mesh->Lz / mesh->nz};
    Elem<double> e;
    head_elem_stack(g.P, H, e);
    return noalloc_head_apply_dot(g, e, Ss, dt, K, x, y, xAx, device, (cudaStream_t)cuda_stream, msg, msg_len);
}

int ht_mixture(double phi, double lambda_s, double lambda_w, double c_s, double c_w, double* lambda, double* cT) {
    if (!lambda || !cT || !(phi >= 0 && phi <= 1)) return HT_EINVAL;
    *lambda = (1.0 - phi) * lambda_s + phi * lambda_w;
    *cT = (1.0 - phi) * c_s + phi * c_w;
    return HT_OK;
}

double ht_specific_storage(double B_poro, double rho_w, double g) { return rho_w * g / B_poro; }

}  // extern "C"
