/*
 * sem_oracle.c -- plain, slow, FP64 CPU oracle for the SEM Q-isosurface render path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package smoke check and the
 * CPU-baseline leg of bench.py load this file.  The CUDA library never calls it, and the
 * two share no code: no header, helper, table or constant generator.
 *
 * What is computed.  The paper renders NekRS spectral-element (SEM) fields in situ
 * (Sec. 1: NekRS is rooted in the spectral element method; Sec. 3.2: the Nek5000/NekRS data
 * model, handed over per step by the DataAdaptor, Listings 2-3).  It does not write out
 * the visualisation arithmetic, so each function below restates the textbook definition
 * it names:
 *   - Gauss-Lobatto-Legendre (GLL) nodes, weights and the collocation derivative matrix D
 *     (Canuto, Hussaini, Quarteroni & Zang, "Spectral Methods", Sec. 2.3; Deville, Fischer &
 *     Mund, "High-Order Methods for Incompressible Fluid Flow", Sec. 2.4);
 *   - the tensor-product derivative of a field on each element and the isoparametric
 *     chain rule (Deville-Fischer-Mund Sec. 4.5);
 *   - the Q-criterion Q = 1/2(|Omega|^2 - |S|^2) = -1/2 sum_ij J_ij J_ji of the velocity
 *     gradient J (Hunt, Wray & Moin 1988);
 *   - marching cubes over the N^3 sub-hexes of each element's GLL lattice (Lorensen &
 *     Cline 1987) with a case table generated here from a face-consistent rule;
 *   - a z-buffer rasteriser with pixel-centre sampling and the top-left fill rule;
 *   - FP64 surface area and divergence-theorem enclosed volume of a triangle soup.
 *
 * Layouts: element e, node n = i + (N+1)(j + (N+1)k); fields f[e*(N+1)^3 + n];
 * coordinates SoA xyz[c*E*(N+1)^3 + e*(N+1)^3 + n].
 *
 * Everything is FP64.  Inputs that the GPU consumes in FP32 are passed here promoted to FP64
 * (exactly), so comparisons of a field against an isovalue decide identically.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared (no FMA contraction, so the
 * x86 and Arm builds give identical results).
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_API __attribute__((visibility("default")))
#define ORC_PI 3.14159265358979323846

#define ORC_MAXT 12 /* triangle slots per marching-cubes case (<= 12 cut edges) */

/* ======================================================================================
 * 1. GLL nodes, weights, derivative matrix                        (Canuto et al. Sec. 2.3)
 * ====================================================================================== */

/* Legendre P_n(x) and P_n'(x) by the three-term recurrence
 *   (n+1) P_{n+1} = (2n+1) x P_n - n P_{n-1},   P'_{n+1} = P'_{n-1} + (2n+1) P_n. */
static void legendre(int N, double x, double *pN, double *dpN, double *pNm1)
{
    double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
    if (N == 0) { *pN = 1.0; *dpN = 0.0; if (pNm1) *pNm1 = 0.0; return; }
    for (int n = 1; n < N; ++n) {
        double p2 = ((2.0 * n + 1.0) * x * p1 - n * p0) / (n + 1.0);
        double d2 = d0 + (2.0 * n + 1.0) * p1;
        p0 = p1; p1 = p2; d0 = d1; d1 = d2;
    }
    *pN = p1; *dpN = d1; if (pNm1) *pNm1 = p0;
}

/* GLL nodes: xi_0 = -1, xi_N = +1, interior nodes = roots of P_N'.  Newton's method on
 * P_N' from Chebyshev-Gauss-Lobatto guesses, with P_N'' taken from Legendre's equation
 * (1-x^2) P'' = 2x P' - N(N+1) P.  Weights w_j = 2 / (N(N+1) P_N(xi_j)^2). */
ORC_API int orc_gll(int N, double *xi, double *w)
{
    if (N < 1 || N > 64) return 1;
    xi[0] = -1.0; xi[N] = 1.0;
    for (int j = 1; j < N; ++j) {
        double x = -cos(ORC_PI * (double)j / (double)N);
        for (int it = 0; it < 100; ++it) {
            double p, dp;
            legendre(N, x, &p, &dp, NULL);
            double d2p = (2.0 * x * dp - N * (N + 1.0) * p) / (1.0 - x * x);
            double dx = dp / d2p;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        xi[j] = x;
    }
    if (w) {
        for (int j = 0; j <= N; ++j) {
            double p, dp;
            legendre(N, xi[j], &p, &dp, NULL);
            w[j] = 2.0 / (N * (N + 1.0) * p * p);
        }
    }
    return 0;
}

/* Collocation derivative matrix on the GLL nodes, D[i*(N+1)+j] = l_j'(xi_i):
 *   D_ij = P_N(xi_i) / (P_N(xi_j) (xi_i - xi_j))  (i != j),
 *   D_00 = -N(N+1)/4,  D_NN = +N(N+1)/4,  else D_ii = 0. */
ORC_API int orc_dmat(int N, const double *xi, double *D)
{
    int NP = N + 1;
    double *P = (double *)malloc(sizeof(double) * NP);
    if (!P) return 3;
    for (int j = 0; j < NP; ++j) { double dp; legendre(N, xi[j], &P[j], &dp, NULL); }
    for (int i = 0; i < NP; ++i)
        for (int j = 0; j < NP; ++j) {
            double v;
            if (i != j) v = P[i] / (P[j] * (xi[i] - xi[j]));
            else if (i == 0) v = -N * (N + 1.0) / 4.0;
            else if (i == N) v = N * (N + 1.0) / 4.0;
            else v = 0.0;
            D[i * NP + j] = v;
        }
    free(P);
    return 0;
}

/* ======================================================================================
 * 2. Tensor-product derivatives and the isoparametric chain rule  (Deville et al. Sec. 4.5)
 * ====================================================================================== */

/* Reference-space derivatives of one element's field f[k][j][i]:
 *   f_r[k][j][i] = sum_m D[i][m] f[k][j][m]
 *   f_s[k][j][i] = sum_m D[j][m] f[k][m][i]
 *   f_t[k][j][i] = sum_m D[k][m] f[m][j][i]                                              */
static void ref_grad(int NP, const double *D, const double *f, double *fr, double *fs, double *ft)
{
    for (int k = 0; k < NP; ++k)
        for (int j = 0; j < NP; ++j)
            for (int i = 0; i < NP; ++i) {
                double a = 0.0, b = 0.0, c = 0.0;
                for (int m = 0; m < NP; ++m) {
                    a += D[i * NP + m] * f[(k * NP + j) * NP + m];
                    b += D[j * NP + m] * f[(k * NP + m) * NP + i];
                    c += D[k * NP + m] * f[(m * NP + j) * NP + i];
                }
                int n = (k * NP + j) * NP + i;
                fr[n] = a; fs[n] = b; ft[n] = c;
            }
}

/* Physical gradient of nf fields on E elements of order N.  For each node the Jacobian
 * J[a][d] = dx_a/dr_d is the reference derivative of the node coordinates; its inverse
 * gives dr_d/dx_a and df/dx_a = sum_d (df/dr_d)(dr_d/dx_a).  Works for any (curved)
 * isoparametric element, not only affine boxes.
 *   fields: nf arrays of E*(N+1)^3;  grad: nf*3 arrays, grad[(q*3+a)*E*NP3 + ...]. */
ORC_API int orc_gradient(int N, int64_t E, const double *xyz, int nf, const double *fields, double *grad)
{
    int NP = N + 1, NP3 = NP * NP * NP;
    int64_t tot = E * (int64_t)NP3;
    double xi[64], D[64 * 64];
    if (N < 1 || N > 63) return 1;
    orc_gll(N, xi, NULL);
    orc_dmat(N, xi, D);
    double *buf = (double *)malloc(sizeof(double) * NP3 * 12);
    if (!buf) return 3;
    double *xr = buf; /* 9 geometric derivatives: [a][d] */
    double *fr = buf + 9 * NP3;
    for (int64_t e = 0; e < E; ++e) {
        for (int a = 0; a < 3; ++a)
            ref_grad(NP, D, xyz + a * tot + e * NP3, xr + (a * 3 + 0) * NP3, xr + (a * 3 + 1) * NP3,
                     xr + (a * 3 + 2) * NP3);
        for (int q = 0; q < nf; ++q) {
            ref_grad(NP, D, fields + q * tot + e * NP3, fr, fr + NP3, fr + 2 * NP3);
            for (int n = 0; n < NP3; ++n) {
                double J[3][3], Ji[3][3];
                for (int a = 0; a < 3; ++a)
                    for (int d = 0; d < 3; ++d) J[a][d] = xr[(a * 3 + d) * NP3 + n];
                double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1])
                           - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0])
                           + J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
                if (det == 0.0) { free(buf); return 4; }
                /* Ji[d][a] = dr_d/dx_a = adj(J)[d][a] / det */
                Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
                Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
                Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
                Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
                Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
                Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
                Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
                Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
                Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
                for (int a = 0; a < 3; ++a) {
                    double g = 0.0;
                    for (int d = 0; d < 3; ++d) g += fr[d * NP3 + n] * Ji[d][a];
                    grad[(q * 3 + a) * tot + e * NP3 + n] = g;
                }
            }
        }
    }
    free(buf);
    return 0;
}

/* ======================================================================================
 * 3. Q-criterion                                                   (Hunt, Wray & Moin 1988)
 *    J_ij = du_i/dx_j,  S = (J+J^T)/2,  Omega = (J-J^T)/2,
 *    Q = 1/2 (|Omega|_F^2 - |S|_F^2) = -1/2 sum_ij J_ij J_ji.
 * ====================================================================================== */
ORC_API int orc_q_from_gradient(int64_t npts, const double *grad /* 9 x npts, [i*3+j] */, double *Q)
{
    for (int64_t p = 0; p < npts; ++p) {
        double s = 0.0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) s += grad[(i * 3 + j) * npts + p] * grad[(j * 3 + i) * npts + p];
        Q[p] = -0.5 * s;
    }
    return 0;
}

ORC_API int orc_qcriterion(int N, int64_t E, const double *xyz, const double *uvw /* 3 fields */, double *Q)
{
    int NP = N + 1;
    int64_t npts = E * (int64_t)NP * NP * NP;
    double *grad = (double *)malloc(sizeof(double) * 9 * (size_t)npts);
    if (!grad) return 3;
    int rc = orc_gradient(N, E, xyz, 3, uvw, grad);
    if (rc == 0) rc = orc_q_from_gradient(npts, grad, Q);
    free(grad);
    return rc;
}

/* ======================================================================================
 * 4. Marching-cubes case table, generated from a face-consistent rule
 *
 * Cell corners v = a + 2b + 4c for offsets (a,b,c) in {0,1}^3 along (i,j,k).  The 12 edges
 * are the corner pairs (lo, hi) differing in one bit, numbered in lexicographic order of
 * (lo, hi).  A corner is inside when f >= iso.  Rule:
 *   (i)   an edge is cut when its ends differ;
 *   (ii)  on each face the cut edges are joined in pairs; on a face with four cut edges
 *         (diagonal inside corners) each inside corner is cut off on its own;
 *   (iii) each face segment P->Q is oriented so that, seen from outside the cell, its
 *         inside corner lies to its left: ((Q-P) x (c-P)) . n_face > 0;
 *   (iv)  segments chain into closed loops (every cut edge lies on two faces);
 *   (v)   loops are taken in order of their lowest edge, each starting at its lowest
 *         edge and fan-triangulated (l0, l_i, l_{i+1}).
 * Step (iii) makes the triangle normal (p1-p0)x(p2-p0) point toward increasing f.
 * Geometric version: segments are oriented with the cross product at the edge midpoints.
 * ====================================================================================== */

static int g_edge_lo[12], g_edge_hi[12];

static void edge_list(void)
{
    int n = 0;
    for (int lo = 0; lo < 8; ++lo)
        for (int hi = lo + 1; hi < 8; ++hi) {
            int x = lo ^ hi;
            if (x == 1 || x == 2 || x == 4) { g_edge_lo[n] = lo; g_edge_hi[n] = hi; ++n; }
        }
}

static int edge_of(int a, int b)
{
    int lo = a < b ? a : b, hi = a < b ? b : a;
    for (int e = 0; e < 12; ++e)
        if (g_edge_lo[e] == lo && g_edge_hi[e] == hi) return e;
    return -1;
}

static void corner_pos(int v, double p[3]) { p[0] = v & 1; p[1] = (v >> 1) & 1; p[2] = (v >> 2) & 1; }

static void edge_mid(int e, double p[3])
{
    double a[3], b[3];
    corner_pos(g_edge_lo[e], a); corner_pos(g_edge_hi[e], b);
    for (int d = 0; d < 3; ++d) p[d] = 0.5 * (a[d] + b[d]);
}

/* +1 if P->Q has corner c on its left seen from outside along normal n, -1 otherwise */
static int seg_side(int eP, int eQ, int c, const double n[3])
{
    double P[3], Q[3], C[3], d[3], w[3], x[3];
    edge_mid(eP, P); edge_mid(eQ, Q); corner_pos(c, C);
    for (int k = 0; k < 3; ++k) { d[k] = Q[k] - P[k]; w[k] = C[k] - P[k]; }
    x[0] = d[1] * w[2] - d[2] * w[1];
    x[1] = d[2] * w[0] - d[0] * w[2];
    x[2] = d[0] * w[1] - d[1] * w[0];
    double s = x[0] * n[0] + x[1] * n[1] + x[2] * n[2];
    return s > 0 ? 1 : -1;
}

/* ntri[256], tri[256*ORC_MAXT*3] (edge indices, -1 padded).  Returns the largest ntri, or a
 * negative value if the rule fails to close a loop (a generator bug). */
ORC_API int orc_mc_table(int *ntri, int *tri)
{
    edge_list();
    int maxt = 0;
    for (int cs = 0; cs < 256; ++cs) {
        int next[12];
        for (int e = 0; e < 12; ++e) next[e] = -1;
        for (int axis = 0; axis < 3; ++axis)
            for (int side = 0; side < 2; ++side) {
                double n[3] = {0, 0, 0};
                n[axis] = side ? 1.0 : -1.0;
                int fc[4], nf = 0;
                for (int v = 0; v < 8; ++v)
                    if (((v >> axis) & 1) == side) fc[nf++] = v;
                /* face edges and their cut status */
                int fe[4], ncut = 0, cut[4];
                int m = 0;
                for (int a = 0; a < 4; ++a)
                    for (int b = a + 1; b < 4; ++b) {
                        int x = fc[a] ^ fc[b];
                        if (x == 1 || x == 2 || x == 4) {
                            int e = edge_of(fc[a], fc[b]);
                            fe[m++] = e;
                            int ia = (cs >> fc[a]) & 1, ib = (cs >> fc[b]) & 1;
                            if (ia != ib) cut[ncut++] = e;
                        }
                    }
                (void)fe;
                if (ncut == 0) continue;
                if (ncut == 2) {
                    int ref = -1;
                    for (int a = 0; a < 4; ++a) if ((cs >> fc[a]) & 1) { ref = fc[a]; break; }
                    int eP = cut[0], eQ = cut[1];
                    if (seg_side(eP, eQ, ref, n) < 0) { int t = eP; eP = eQ; eQ = t; }
                    if (next[eP] != -1) return -1;
                    next[eP] = eQ;
                } else if (ncut == 4) {
                    for (int a = 0; a < 4; ++a) {
                        int c = fc[a];
                        if (!((cs >> c) & 1)) continue;
                        int adj[2], na = 0;
                        for (int b = 0; b < 4; ++b) {
                            int x = c ^ fc[b];
                            if (x == 1 || x == 2 || x == 4) adj[na++] = edge_of(c, fc[b]);
                        }
                        int eP = adj[0], eQ = adj[1];
                        if (seg_side(eP, eQ, c, n) < 0) { int t = eP; eP = eQ; eQ = t; }
                        if (next[eP] != -1) return -1;
                        next[eP] = eQ;
                    }
                } else {
                    return -2;
                }
            }
        /* chain loops, lowest unused edge first */
        int used[12] = {0}, nt = 0;
        for (int k = 0; k < ORC_MAXT * 3; ++k) tri[cs * ORC_MAXT * 3 + k] = -1;
        for (int e0 = 0; e0 < 12; ++e0) {
            if (next[e0] == -1 || used[e0]) continue;
            int loop[13], len = 0, e = e0;
            while (!used[e]) {
                if (e < 0 || len >= 12) return -3;
                used[e] = 1; loop[len++] = e; e = next[e];
            }
            if (e != e0) return -4;
            for (int q = 1; q + 1 < len; ++q) {
                tri[(cs * ORC_MAXT + nt) * 3 + 0] = loop[0];
                tri[(cs * ORC_MAXT + nt) * 3 + 1] = loop[q];
                tri[(cs * ORC_MAXT + nt) * 3 + 2] = loop[q + 1];
                ++nt;
            }
        }
        ntri[cs] = nt;
        if (nt > maxt) maxt = nt;
    }
    return maxt;
}

ORC_API int orc_mc_maxt(void) { return ORC_MAXT; }

/* ======================================================================================
 * 5. Marching cubes over the N^3 sub-hexes of each element          (Lorensen & Cline 1987)
 *
 * Cell (i,j,k), i,j,k in [0,N), corner v -> node (i+a, j+b, k+c).  case = sum_v [f_v>=iso] 2^v.
 * Cut edge (lo,hi): t = (iso - f_lo)/(f_hi - f_lo), p = p_lo + t (p_hi - p_lo).
 * Output order: element, cell index i + N(j + Nk), table order.
 *   cases:     optional, E*N^3 bytes
 *   elem_ntri: optional, E triangle counts
 *   tris:      cap*9 doubles (v0xyz v1xyz v2xyz); tri_elem: cap ints (both optional)
 * Returns 0, or 2 when more than cap triangles were found (*ntri_out = required count).
 * ====================================================================================== */
ORC_API int orc_isosurface(int N, int64_t E, const double *xyz, const double *f, double iso,
                           uint8_t *cases, int64_t *elem_ntri, int64_t cap, double *tris,
                           int32_t *tri_elem, int64_t *ntri_out)
{
    static int T_n[256], T_t[256 * ORC_MAXT * 3];
    static int have = 0;
    if (!have) { if (orc_mc_table(T_n, T_t) < 0) return 5; have = 1; }
    int NP = N + 1, NP3 = NP * NP * NP, N3 = N * N * N;
    int64_t tot = E * (int64_t)NP3;
    int64_t nt = 0;
    for (int64_t e = 0; e < E; ++e) {
        const double *fe = f + e * NP3;
        int64_t ne = 0;
        for (int k = 0; k < N; ++k)
            for (int j = 0; j < N; ++j)
                for (int i = 0; i < N; ++i) {
                    int node[8], cs = 0;
                    for (int v = 0; v < 8; ++v) {
                        node[v] = (i + (v & 1)) + NP * ((j + ((v >> 1) & 1)) + NP * (k + ((v >> 2) & 1)));
                        if (fe[node[v]] >= iso) cs |= 1 << v;
                    }
                    if (cases) cases[e * N3 + i + N * (j + N * k)] = (uint8_t)cs;
                    for (int q = 0; q < T_n[cs]; ++q) {
                        if (nt < cap && tris) {
                            for (int s = 0; s < 3; ++s) {
                                int ed = T_t[(cs * ORC_MAXT + q) * 3 + s];
                                int lo = g_edge_lo[ed], hi = g_edge_hi[ed];
                                double fa = fe[node[lo]], fb = fe[node[hi]];
                                double t = (iso - fa) / (fb - fa);
                                for (int c = 0; c < 3; ++c) {
                                    double pa = xyz[c * tot + e * NP3 + node[lo]];
                                    double pb = xyz[c * tot + e * NP3 + node[hi]];
                                    tris[nt * 9 + s * 3 + c] = pa + t * (pb - pa);
                                }
                            }
                            if (tri_elem) tri_elem[nt] = (int32_t)e;
                        }
                        ++nt; ++ne;
                    }
                }
        if (elem_ntri) elem_ntri[e] = ne;
    }
    *ntri_out = nt;
    return nt > cap ? 2 : 0;
}

/* ======================================================================================
 * 6. Z-buffer rasteriser (headless RGBA8 + depth)
 *
 * View basis from eye/center/up: f = unit(center-eye), s = unit(f x up), u = s x f;
 * view coordinates xv = s.(p-eye), yv = u.(p-eye), zv = f.(p-eye).
 * Orthographic:  x_ndc = xv/(half_h*aspect), y_ndc = yv/half_h, z_ndc = (zv-zn)/(zf-zn).
 * Perspective:   x_ndc = xv/(zv tan(fovy/2) aspect), y_ndc = yv/(zv tan(fovy/2)),
 *                z_ndc = zf/(zf-zn) (1 - zn/zv).
 * A triangle with any vertex at zv <= znear or zv >= zfar is dropped.
 * Screen: sx = (x_ndc+1)/2 W, sy = (1-y_ndc)/2 H; pixel (px,py) samples (px+.5, py+.5).
 * Coverage: edge functions of the triangle made clockwise on screen (y down); a sample
 * exactly on an edge is covered only for top edges (dy == 0, dx > 0) and left edges
 * (dy < 0).  Zero-area triangles are skipped; no back-face culling.  Depth is z_ndc
 * interpolated barycentrically in screen space.  The smallest (depth, triangle index)
 * wins.  Shading: c = rgb[seg] (0.15 + 0.85 |n.l|), n = unit((p1-p0)x(p2-p0)), l = -f;
 * rgba8 = floor(clamp(c,0,1)*255 + 0.5), alpha 255; background (0,0,0,0), depth 1.
 * ====================================================================================== */

static void cross3(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void unit3(double a[3]) { double n = sqrt(dot3(a, a)); a[0] /= n; a[1] /= n; a[2] /= n; }

static int top_left(double ax, double ay, double bx, double by)
{
    double dx = bx - ax, dy = by - ay;
    return (dy < 0.0) || (dy == 0.0 && dx > 0.0);
}

ORC_API int orc_render(const double *tris, int64_t ntri, const int64_t *seg_end, int nseg,
                       const double *seg_rgb, int ortho, const double *eye, const double *center,
                       const double *up, double fovy_deg, double half_h, double znear, double zfar,
                       int W, int H, uint8_t *rgba, double *depth, int64_t *winner)
{
    double f[3], s[3], u[3];
    for (int k = 0; k < 3; ++k) f[k] = center[k] - eye[k];
    unit3(f);
    cross3(f, up, s); unit3(s);
    cross3(s, f, u);
    double aspect = (double)W / (double)H;
    double th = tan(0.5 * fovy_deg * ORC_PI / 180.0);
    int64_t npx = (int64_t)W * H;
    int64_t *best = winner ? winner : (int64_t *)malloc(sizeof(int64_t) * npx);
    double *bz = (double *)malloc(sizeof(double) * npx);
    if (!best || !bz) return 3;
    for (int64_t p = 0; p < npx; ++p) { best[p] = -1; bz[p] = INFINITY; }

    for (int64_t t = 0; t < ntri; ++t) {
        double sx[3], sy[3], sz[3];
        int drop = 0;
        for (int v = 0; v < 3; ++v) {
            double d[3];
            for (int k = 0; k < 3; ++k) d[k] = tris[t * 9 + v * 3 + k] - eye[k];
            double xv = dot3(s, d), yv = dot3(u, d), zv = dot3(f, d);
            if (!(zv > znear && zv < zfar)) { drop = 1; break; }
            double xn, yn, zn;
            if (ortho) {
                xn = xv / (half_h * aspect); yn = yv / half_h; zn = (zv - znear) / (zfar - znear);
            } else {
                xn = xv / (zv * th * aspect); yn = yv / (zv * th); zn = zfar / (zfar - znear) * (1.0 - znear / zv);
            }
            sx[v] = (xn + 1.0) * 0.5 * W;
            sy[v] = (1.0 - yn) * 0.5 * H;
            sz[v] = zn;
        }
        if (drop) continue;
        double area = (sx[1] - sx[0]) * (sy[2] - sy[0]) - (sx[2] - sx[0]) * (sy[1] - sy[0]);
        if (area == 0.0 || isnan(area)) continue;
        if (area < 0.0) { /* make clockwise on screen (y down) */
            double tx = sx[1], ty = sy[1], tz = sz[1];
            sx[1] = sx[2]; sy[1] = sy[2]; sz[1] = sz[2];
            sx[2] = tx; sy[2] = ty; sz[2] = tz;
            area = -area;
        }
        double mnx = fmin(sx[0], fmin(sx[1], sx[2])), mxx = fmax(sx[0], fmax(sx[1], sx[2]));
        double mny = fmin(sy[0], fmin(sy[1], sy[2])), mxy = fmax(sy[0], fmax(sy[1], sy[2]));
        int x0 = (int)fmax(0.0, floor(mnx) - 1), x1 = (int)fmin(W - 1.0, ceil(mxx) + 1);
        int y0 = (int)fmax(0.0, floor(mny) - 1), y1 = (int)fmin(H - 1.0, ceil(mxy) + 1);
        int tl0 = top_left(sx[0], sy[0], sx[1], sy[1]);
        int tl1 = top_left(sx[1], sy[1], sx[2], sy[2]);
        int tl2 = top_left(sx[2], sy[2], sx[0], sy[0]);
        for (int py = y0; py <= y1; ++py)
            for (int px = x0; px <= x1; ++px) {
                double cx = px + 0.5, cy = py + 0.5;
                double e0 = (sx[1] - sx[0]) * (cy - sy[0]) - (sy[1] - sy[0]) * (cx - sx[0]);
                double e1 = (sx[2] - sx[1]) * (cy - sy[1]) - (sy[2] - sy[1]) * (cx - sx[1]);
                double e2 = (sx[0] - sx[2]) * (cy - sy[2]) - (sy[0] - sy[2]) * (cx - sx[2]);
                int in = (e0 > 0.0 || (e0 == 0.0 && tl0)) && (e1 > 0.0 || (e1 == 0.0 && tl1))
                      && (e2 > 0.0 || (e2 == 0.0 && tl2));
                if (!in) continue;
                double z = (e1 * sz[0] + e2 * sz[1] + e0 * sz[2]) / area;
                int64_t p = (int64_t)py * W + px;
                if (z < bz[p] || (z == bz[p] && t < best[p])) { bz[p] = z; best[p] = t; }
            }
    }

    double l[3] = {-f[0], -f[1], -f[2]};
    for (int64_t p = 0; p < npx; ++p) {
        int64_t t = best[p];
        if (t < 0) {
            rgba[p * 4 + 0] = rgba[p * 4 + 1] = rgba[p * 4 + 2] = rgba[p * 4 + 3] = 0;
            depth[p] = 1.0;
            continue;
        }
        int sg = 0;
        while (sg < nseg - 1 && t >= seg_end[sg]) ++sg;
        double a[3], b[3], n[3];
        for (int k = 0; k < 3; ++k) {
            a[k] = tris[t * 9 + 3 + k] - tris[t * 9 + k];
            b[k] = tris[t * 9 + 6 + k] - tris[t * 9 + k];
        }
        cross3(a, b, n);
        double nn = sqrt(dot3(n, n));
        double shade = nn > 0.0 ? 0.15 + 0.85 * fabs(dot3(n, l)) / nn : 0.15;
        for (int k = 0; k < 3; ++k) {
            double c = seg_rgb[sg * 3 + k] * shade;
            c = c < 0.0 ? 0.0 : (c > 1.0 ? 1.0 : c);
            rgba[p * 4 + k] = (uint8_t)floor(c * 255.0 + 0.5);
        }
        rgba[p * 4 + 3] = 255;
        depth[p] = bz[p];
    }
    if (!winner) free(best);
    free(bz);
    return 0;
}

/* ======================================================================================
 * 7. FP64 global reductions of a triangle soup
 *    area = sum |(p1-p0)x(p2-p0)|/2;  volume = (1/3) sum pbar.n A = sum p0.(p1 x p2)/6
 *    (divergence theorem with div x = 3; positive when normals point out of the region).
 * ====================================================================================== */
ORC_API int orc_surface_measures(const double *tris, int64_t ntri, double *area, double *volume)
{
    double A = 0.0, V = 0.0;
    for (int64_t t = 0; t < ntri; ++t) {
        const double *p = tris + t * 9;
        double a[3], b[3], n[3], c[3];
        for (int k = 0; k < 3; ++k) { a[k] = p[3 + k] - p[k]; b[k] = p[6 + k] - p[k]; }
        cross3(a, b, n);
        A += 0.5 * sqrt(dot3(n, n));
        cross3(p + 3, p + 6, c);
        V += dot3(p, c) / 6.0;
    }
    *area = A; *volume = V;
    return 0;
}
