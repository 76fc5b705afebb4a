// sem_api.cu -- C ABI of libsem: contexts, meshes, argument checking, host-side table
// generators (GLL nodes / derivative matrix, marching-cubes case table).
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "sem_internal.cuh"

#define SEM_ABI_VERSION 1

static thread_local std::string g_create_err;

sem_status sem_fail(sem_ctx *ctx, sem_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx)
        ctx->err = buf;
    else
        g_create_err = buf;
    return st;
}

sem_status sem_cuda(sem_ctx *ctx, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return SEM_OK;
    cudaGetLastError();  // clear a non-sticky error
    return sem_fail(ctx, e == cudaErrorMemoryAllocation ? SEM_ERR_OOM : SEM_ERR_CUDA, "%s: %s (%s)", what,
                    cudaGetErrorString(e), cudaGetErrorName(e));
}

sem_status sem_scratch(sem_ctx *ctx, int slot, size_t bytes, void **out)
{
    if (bytes == 0) bytes = 256;
    if (ctx->scratch_bytes[slot] < bytes) {
        size_t nb = bytes + bytes / 4 + 4096;
        if (ctx->scratch[slot]) {
            SEM_CU(ctx, cudaStreamSynchronize(ctx->stream));
            SEM_CU(ctx, cudaFree(ctx->scratch[slot]));
            ctx->mem_add(-(int64_t)ctx->scratch_bytes[slot]);
            ctx->scratch[slot] = nullptr;
            ctx->scratch_bytes[slot] = 0;
        }
        SEM_CU(ctx, cudaMalloc(&ctx->scratch[slot], nb));
        ctx->scratch_bytes[slot] = nb;
        ctx->mem_add((int64_t)nb);
    }
    *out = ctx->scratch[slot];
    return SEM_OK;
}

sem_status sem_scratch_nogrow_in_capture(sem_ctx *ctx, int slot, size_t bytes, void **out)
{
    if (ctx->scratch_bytes[slot] < (bytes ? bytes : 256)) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        SEM_CU(ctx, cudaStreamIsCapturing(ctx->stream, &cs));
        if (cs != cudaStreamCaptureStatusNone)
            return sem_fail(ctx, SEM_ERR_CAPACITY,
                            "scratch arena %d too small while the stream is captured (%zu < %zu bytes): make the "
                            "same call once before capturing",
                            slot, ctx->scratch_bytes[slot], bytes);
    }
    return sem_scratch(ctx, slot, bytes, out);
}

// ==========================================================================================
// GLL nodes and derivative matrix (host, FP64).
//
// Interior GLL nodes are the zeros of P_N' = ((N+1)/2) P^{(1,1)}_{N-1}, the Jacobi polynomial
// with alpha = beta = 1 (Canuto et al., Spectral Methods, Sec. 2.3).  They are found by
// Newton's method on P^{(1,1)}_{N-1}, evaluated with its three-term recurrence
//   2n(n+2) P_n = (2n+1)(2n+2) x P_{n-1} - n(2n+2) P_{n-2},  P_0 = 1, P_1 = 2x.
// D is the derivative of the Lagrange basis in barycentric form (Berrut & Trefethen 2004):
//   lambda_j = 1 / prod_{k != j} (x_j - x_k),  D_ij = (lambda_j / lambda_i) / (x_i - x_j),
//   D_ii = -sum_{j != i} D_ij.
// ==========================================================================================
static void jacobi11(int n, double x, double *p, double *dp)
{
    double p0 = 1.0, p1 = 2.0 * x, d0 = 0.0, d1 = 2.0;
    if (n == 0) {
        *p = 1.0;
        *dp = 0.0;
        return;
    }
    for (int k = 2; k <= n; ++k) {
        double a = (2.0 * k + 1.0) * (2.0 * k + 2.0), b = k * (2.0 * k + 2.0), c = 2.0 * k * (k + 2.0);
        double p2 = (a * x * p1 - b * p0) / c;
        double d2 = (a * (p1 + x * d1) - b * d0) / c;
        p0 = p1;
        p1 = p2;
        d0 = d1;
        d1 = d2;
    }
    *p = p1;
    *dp = d1;
}

static void gll_nodes(int N, double *x)
{
    x[0] = -1.0;
    x[N] = 1.0;
    for (int j = 1; j < N; ++j) {
        double t = -cos(M_PI * j / N);
        for (int it = 0; it < 200; ++it) {
            double p, dp;
            jacobi11(N - 1, t, &p, &dp);
            double step = p / dp;
            t -= step;
            if (fabs(step) < 1e-17) break;
        }
        x[j] = t;
    }
}

static void gll_dmat(int N, const double *x, double *D)
{
    int NP = N + 1;
    std::vector<double> lam(NP);
    for (int j = 0; j < NP; ++j) {
        double pr = 1.0;
        for (int k = 0; k < NP; ++k)
            if (k != j) pr *= (x[j] - x[k]);
        lam[j] = 1.0 / pr;
    }
    for (int i = 0; i < NP; ++i) {
        double diag = 0.0;
        for (int j = 0; j < NP; ++j) {
            if (j == i) continue;
            double v = (lam[j] / lam[i]) / (x[i] - x[j]);
            D[i * NP + j] = v;
            diag -= v;
        }
        D[i * NP + i] = diag;
    }
}

// ==========================================================================================
// Marching-cubes case table (host).  Corners v = a + 2b + 4c, edges = corner pairs differing
// in one bit, numbered lexicographically by (lower, upper) corner.  Rule: on every face, walk
// the corners counter-clockwise as seen from outside the cell; each maximal run of inside
// corners (f >= iso) is bounded by an entry edge (outside -> inside) and an exit edge
// (inside -> outside); the face contributes the segment exit -> entry.  A face with
// diagonal inside corners has two runs, so each inside corner is cut off on its own, and two
// cells sharing a face derive the same segments (crack-free).  Segments chain into closed
// loops (each cut edge lies on two faces); loops are taken by their lowest edge, start at it
// and are fan-triangulated.  The walk direction makes (p1-p0)x(p2-p0) point toward
// increasing f (Lorensen & Cline 1987 for the method; the table is generated, not copied).
// ==========================================================================================
static int mc_build(int32_t *ntri, int8_t *edges)
{
    int eid[8][8];
    for (int a = 0; a < 8; ++a)
        for (int b = 0; b < 8; ++b) eid[a][b] = -1;
    int ne = 0;
    for (int lo = 0; lo < 8; ++lo)
        for (int hi = lo + 1; hi < 8; ++hi) {
            int x = lo ^ hi;
            if (x == 1 || x == 2 || x == 4) {
                eid[lo][hi] = eid[hi][lo] = ne++;
            }
        }
    static const int ccw_pos[4][2] = {{0, 0}, {1, 0}, {1, 1}, {0, 1}};
    int maxt = 0;
    for (int cs = 0; cs < 256; ++cs) {
        int succ[12];
        for (int e = 0; e < 12; ++e) succ[e] = -1;
        for (int d = 0; d < 3; ++d) {
            int a = (d + 1) % 3, b = (d + 2) % 3;  // e_a x e_b = e_d
            for (int side = 0; side < 2; ++side) {
                int cyc[4];
                for (int m = 0; m < 4; ++m) {
                    // counter-clockwise about the outward normal: +e_d keeps the (a,b) order,
                    // -e_d reverses it
                    int mm = side ? m : (4 - m) % 4;
                    cyc[m] = (side << d) | (ccw_pos[mm][0] << a) | (ccw_pos[mm][1] << b);
                }
                for (int m = 0; m < 4; ++m) {
                    int prev = cyc[(m + 3) % 4], cur = cyc[m];
                    bool pin = (cs >> prev) & 1, cin = (cs >> cur) & 1;
                    if (pin || !cin) continue;  // not the first corner of an inside run
                    int e_in = eid[prev][cur];
                    int q = m;
                    while ((cs >> cyc[(q + 1) % 4]) & 1) q = (q + 1) % 4;
                    int e_out = eid[cyc[q]][cyc[(q + 1) % 4]];
                    if (succ[e_out] != -1) return -1;
                    succ[e_out] = e_in;
                }
            }
        }
        bool seen[12] = {false};
        int nt = 0;
        for (int k = 0; k < SEM_MC_MAXT * 3; ++k) edges[cs * SEM_MC_MAXT * 3 + k] = -1;
        for (int e0 = 0; e0 < 12; ++e0) {
            if (succ[e0] < 0 || seen[e0]) continue;
            int loop[12], len = 0;
            for (int e = e0; !seen[e]; e = succ[e]) {
                if (succ[e] < 0 || len == 12) return -2;
                seen[e] = true;
                loop[len++] = e;
            }
            for (int q = 1; q + 1 < len; ++q) {
                int8_t *t = edges + (cs * SEM_MC_MAXT + nt) * 3;
                t[0] = (int8_t)loop[0];
                t[1] = (int8_t)loop[q];
                t[2] = (int8_t)loop[q + 1];
                ++nt;
            }
        }
        ntri[cs] = nt;
        if (nt > maxt) maxt = nt;
    }
    return maxt;
}

// ==========================================================================================
// C ABI
// ==========================================================================================
extern "C" {

int sem_version(void) { return SEM_ABI_VERSION; }

int sem_mc_table(int32_t *ntri, int8_t *edges)
{
    if (!ntri || !edges) return -100;
    return mc_build(ntri, edges);
}

sem_status sem_gll(int N, double *xi, double *D)
{
    if (N < 1 || N > SEM_MAX_ORDER || !xi) return SEM_ERR_ARG;
    gll_nodes(N, xi);
    if (D) gll_dmat(N, xi, D);
    return SEM_OK;
}

const char *sem_last_error(const sem_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_err.c_str(); }

static sem_status upload_tables(sem_ctx *ctx)
{
    const int MP = SEM_MAX_ORDER + 1;
    std::vector<float> D_all((size_t)(SEM_MAX_ORDER + 1) * MP * MP, 0.f), s_all((size_t)(SEM_MAX_ORDER + 1) * MP, 0.f);
    double x[MP], D[MP * MP];
    for (int N = 1; N <= SEM_MAX_ORDER; ++N) {
        int NP = N + 1;
        gll_nodes(N, x);
        gll_dmat(N, x, D);
        for (int i = 0; i < NP; ++i) {
            s_all[(size_t)N * MP + i] = (float)((x[i] + 1.0) * 0.5);
            for (int j = 0; j < NP; ++j) D_all[((size_t)N * MP + i) * MP + j] = (float)D[i * NP + j];
        }
        s_all[(size_t)N * MP + 0] = 0.f;
        s_all[(size_t)N * MP + N] = 1.f;
    }
    int32_t ntri[256];
    std::vector<int8_t> edges(256 * SEM_MC_MAXT * 3);
    int mx = mc_build(ntri, edges.data());
    if (mx < 0 || mx > 5) return sem_fail(ctx, SEM_ERR_CUDA, "marching-cubes table generator failed (%d)", mx);
    SEM_TRY(qcrit_upload_tables(ctx, D_all.data(), s_all.data()));
    SEM_TRY(iso_upload_tables(ctx, s_all.data(), ntri, edges.data()));
    return SEM_OK;
}

sem_status sem_create(int device, void *stream, sem_ctx **out)
{
    if (!out) return sem_fail(nullptr, SEM_ERR_ARG, "sem_create: out is NULL");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0)
        return sem_fail(nullptr, SEM_ERR_CUDA, "sem_create: no CUDA device (%s)", cudaGetErrorString(e));
    if (device < 0 || device >= ndev) return sem_fail(nullptr, SEM_ERR_ARG, "sem_create: bad device %d", device);
    sem_ctx *ctx = new sem_ctx();
    ctx->device = device;
    ctx->stream = (cudaStream_t)stream;
    sem_status st = SEM_OK;
    do {
        if ((st = sem_cuda(ctx, cudaSetDevice(device), "cudaSetDevice")) != SEM_OK) break;
        cudaDeviceProp prop;
        if ((st = sem_cuda(ctx, cudaGetDeviceProperties(&prop, device), "cudaGetDeviceProperties")) != SEM_OK) break;
        if (prop.major * 10 + prop.minor < 100) {
            st = sem_fail(ctx, SEM_ERR_UNSUPPORTED, "device %d is sm_%d%d; this build targets sm_103a", device,
                          prop.major, prop.minor);
            break;
        }
        ctx->sm_count = prop.multiProcessorCount;
        if ((st = sem_cuda(ctx, cudaMalloc(&ctx->d_flag, 64), "cudaMalloc(flag)")) != SEM_OK) break;
        ctx->mem_add(64);
        if ((st = sem_cuda(ctx, cudaMemset(ctx->d_flag, 0, 64), "cudaMemset(flag)")) != SEM_OK) break;
        if ((st = sem_cuda(ctx, cudaMallocHost(&ctx->h_pinned, 16 * sizeof(int64_t)), "cudaMallocHost")) != SEM_OK)
            break;
        if ((st = sem_cuda(ctx, cudaMallocHost(&ctx->h_pinned_d, 4 * sizeof(double)), "cudaMallocHost")) != SEM_OK)
            break;
        if ((st = upload_tables(ctx)) != SEM_OK) break;
        if ((st = iso_noalloc_prepare(ctx)) != SEM_OK) break;
        if ((st = sem_cuda(ctx, cudaDeviceSynchronize(), "cudaDeviceSynchronize")) != SEM_OK) break;
    } while (0);
    if (st != SEM_OK) {
        g_create_err = ctx->err;
        sem_destroy(ctx);
        return st;
    }
    *out = ctx;
    return SEM_OK;
}

void sem_destroy(sem_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (auto &r : ctx->trace) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (cudaEvent_t ev : ctx->trace_pool) cudaEventDestroy(ev);
    if (ctx->aux) {
        cudaStreamSynchronize(ctx->aux);
        cudaStreamDestroy(ctx->aux);
    }
    for (cudaEvent_t ev : {ctx->ev_fork, ctx->ev_qseg, ctx->ev_join})
        if (ev) cudaEventDestroy(ev);
    render_frame_free(ctx);
    for (int s = 0; s < SCR_COUNT; ++s)
        if (ctx->scratch[s]) cudaFree(ctx->scratch[s]);
    if (ctx->d_flag) cudaFree(ctx->d_flag);
    for (int s = 0; s < 3; ++s)
        if (ctx->tc_A[s]) cudaFree(ctx->tc_A[s]);
    if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
    if (ctx->h_pinned_d) cudaFreeHost(ctx->h_pinned_d);
    delete ctx;
}

// ------------------------------------------------------------------------------------------
// Kernel trace
// ------------------------------------------------------------------------------------------
TraceScope::TraceScope(sem_ctx *c, const char *name) : ctx(c)
{
    if (!c->trace_on) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    sem_ctx::TraceRec r{name, nullptr, nullptr};
    for (cudaEvent_t *ev : {&r.a, &r.b}) {
        if (!c->trace_pool.empty()) {
            *ev = c->trace_pool.back();
            c->trace_pool.pop_back();
        } else if (cudaEventCreate(ev) != cudaSuccess) {
            return;  // tracing is best effort: an event that cannot be made skips this launch
        }
    }
    if (cudaEventRecord(r.a, c->stream) != cudaSuccess) return;
    c->trace.push_back(r);
    idx = (int)c->trace.size() - 1;
}

TraceScope::~TraceScope()
{
    if (idx >= 0) cudaEventRecord(ctx->trace[idx].b, ctx->stream);
}

sem_status sem_memory(sem_ctx *ctx, int64_t *in_use, int64_t *peak)
{
    if (!ctx || !in_use || !peak) return SEM_ERR_ARG;
    *in_use = ctx->mem_now;
    *peak = ctx->mem_peak;
    return SEM_OK;
}

sem_status sem_trace_enable(sem_ctx *ctx, int on)
{
    if (!ctx) return SEM_ERR_ARG;
    ctx->trace_on = on != 0;
    return SEM_OK;
}

sem_status sem_trace_collect(sem_ctx *ctx, int *n_kernels)
{
    if (!ctx || !n_kernels) return SEM_ERR_ARG;
    SEM_CU(ctx, cudaSetDevice(ctx->device));
    ctx->trace_sum.clear();
    for (auto &r : ctx->trace) {
        SEM_CU(ctx, cudaEventSynchronize(r.b));
        float ms = 0.f;
        SEM_CU(ctx, cudaEventElapsedTime(&ms, r.a, r.b));
        size_t k = 0;
        while (k < ctx->trace_sum.size() && strcmp(ctx->trace_sum[k].name, r.name) != 0) ++k;
        if (k == ctx->trace_sum.size()) ctx->trace_sum.push_back({r.name, 0.0, 0});
        ctx->trace_sum[k].ms += ms;
        ctx->trace_sum[k].launches += 1;
        ctx->trace_pool.push_back(r.a);
        ctx->trace_pool.push_back(r.b);
    }
    ctx->trace.clear();
    *n_kernels = (int)ctx->trace_sum.size();
    return SEM_OK;
}

sem_status sem_trace_entry(sem_ctx *ctx, int k, const char **name, double *total_ms, int64_t *launches)
{
    if (!ctx || !name || !total_ms || !launches) return SEM_ERR_ARG;
    if (k < 0 || k >= (int)ctx->trace_sum.size())
        return sem_fail(ctx, SEM_ERR_ARG, "sem_trace_entry: index %d outside [0, %d)", k, (int)ctx->trace_sum.size());
    *name = ctx->trace_sum[k].name;
    *total_ms = ctx->trace_sum[k].ms;
    *launches = ctx->trace_sum[k].launches;
    return SEM_OK;
}

sem_status sem_set_stream(sem_ctx *ctx, void *stream)
{
    if (!ctx) return SEM_ERR_ARG;
    ctx->stream = (cudaStream_t)stream;
    return SEM_OK;
}

sem_status sem_debug_set_wait_limit(sem_ctx *ctx, int64_t polls)
{
    if (!ctx) return SEM_ERR_ARG;
    ctx->wait_limit = polls < 0 ? SEM_WAIT_LIMIT : (long long)polls;
    return SEM_OK;
}

sem_status sem_synchronize(sem_ctx *ctx)
{
    if (!ctx) return SEM_ERR_ARG;
    SEM_CU(ctx, cudaSetDevice(ctx->device));
    int flag = 0;
    SEM_CU(ctx, cudaMemcpyAsync(&flag, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    SEM_CU(ctx, cudaStreamSynchronize(ctx->stream));
    if (flag) {
        SEM_CU(ctx, cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), ctx->stream));
        SEM_CU(ctx, cudaStreamSynchronize(ctx->stream));
        if (flag & (1 << SEM_ERR_TIMEOUT))
            return sem_fail(ctx, SEM_ERR_TIMEOUT, "a bounded device-side wait ran out (flag 0x%x)", flag);
        if (flag & (1 << SEM_ERR_ARG))
            return sem_fail(ctx, SEM_ERR_ARG, "a kernel found an argument out of range, e.g. a sample index (flag 0x%x)",
                            flag);
        if (flag & (1 << SEM_ERR_CAPACITY))
            return sem_fail(ctx, SEM_ERR_CAPACITY,
                            "an asynchronous call found more triangles than its buffer holds (flag 0x%x)", flag);
        return sem_fail(ctx, SEM_ERR_CUDA, "device-side failure flag 0x%x", flag);
    }
    return SEM_OK;
}

sem_status sem_load_mesh(sem_ctx *ctx, int N, int64_t E, const double *xyz, sem_mesh **out)
{
    if (!ctx) return SEM_ERR_ARG;
    if (!out) return sem_fail(ctx, SEM_ERR_ARG, "sem_load_mesh: out is NULL");
    *out = nullptr;
    if (N < 1 || N > SEM_MAX_ORDER) return sem_fail(ctx, SEM_ERR_ARG, "sem_load_mesh: N=%d outside [1,%d]", N, SEM_MAX_ORDER);
    if (E < 0 || E > (int64_t)1 << 31) return sem_fail(ctx, SEM_ERR_ARG, "sem_load_mesh: bad E=%lld", (long long)E);
    if (E > 0 && !xyz) return sem_fail(ctx, SEM_ERR_ARG, "sem_load_mesh: xyz is NULL");
    const int NP = N + 1, NP3 = NP * NP * NP;
    double xi[SEM_MAX_ORDER + 1], D[(SEM_MAX_ORDER + 1) * (SEM_MAX_ORDER + 1)];
    gll_nodes(N, xi);
    gll_dmat(N, xi, D);
    std::vector<float4> lo(E), hi(E), g(E);
    const int64_t tot = E * NP3;
    for (int64_t q = 0; q < 3 * tot; ++q)
        if (!isfinite(xyz[q])) return sem_fail(ctx, SEM_ERR_ARG, "sem_load_mesh: coordinate %lld is not finite", (long long)q);
    // axis-aligned affine boxes (x = x0 + (xi + 1)/2 (x1 - x0) along each axis, to 1e-9
    // relative) take the fast path; any other element makes the whole mesh general
    bool curved = false;
    for (int64_t e = 0; e < E && !curved; ++e) {
        const double *X = xyz + e * NP3, *Y = xyz + tot + e * NP3, *Z = xyz + 2 * tot + e * NP3;
        const double a[3] = {X[0], Y[0], Z[0]};
        const double b[3] = {X[N], Y[N * NP], Z[N * NP * NP]};
        for (int d = 0; d < 3 && !curved; ++d) curved = !(b[d] != a[d]);  // zero extent: degenerate
        for (int n = 0; n < NP3 && !curved; ++n) {
            const int idx[3] = {n % NP, (n / NP) % NP, n / (NP * NP)};
            const double *P[3] = {X, Y, Z};
            for (int d = 0; d < 3 && !curved; ++d) {
                const double expect = a[d] + (xi[idx[d]] + 1.0) * 0.5 * (b[d] - a[d]);
                curved = !(fabs(P[d][n] - expect) <= 1e-9 * (fabs(b[d] - a[d]) + fabs(a[d])));
            }
        }
    }
    std::vector<float> geo, xyzn;
    if (curved) {
        // per node: Jacobian J[c][d] = d x_c / d r_d = sum_m D[idx_d][m] x_c(node with idx_d = m),
        // its inverse G[d][j] = d r_d / d x_j (FP64, cofactors); a non-positive or non-finite
        // determinant is an inverted or degenerate element
        geo.resize(9 * (size_t)tot);
        xyzn.resize(3 * (size_t)tot);
        const int stride[3] = {1, NP, NP * NP};
        for (int64_t e = 0; e < E; ++e) {
            double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
            for (int n = 0; n < NP3; ++n) {
                const int idx[3] = {n % NP, (n / NP) % NP, n / (NP * NP)};
                double J[3][3];
                for (int c = 0; c < 3; ++c) {
                    const double *Xc = xyz + c * tot + e * NP3;
                    for (int d = 0; d < 3; ++d) {
                        const int base = n - idx[d] * stride[d];
                        double acc = 0.0;
                        for (int m2 = 0; m2 < NP; ++m2) acc += D[idx[d] * NP + m2] * Xc[base + m2 * stride[d]];
                        J[c][d] = acc;
                    }
                    mn[c] = fmin(mn[c], Xc[n]);
                    mx[c] = fmax(mx[c], Xc[n]);
                    xyzn[c * tot + e * NP3 + n] = (float)Xc[n];
                }
                const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
                const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
                const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
                const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
                if (!(det > 0.0) || !isfinite(det))
                    return sem_fail(ctx, SEM_ERR_ARG,
                                    "sem_load_mesh: element %lld is inverted or degenerate at node %d (det J = %g)",
                                    (long long)e, n, det);
                // G = J^-1 = adj(J) / det, G[d][j]
                double G[3][3];
                G[0][0] = c00 / det;
                G[1][0] = c01 / det;
                G[2][0] = c02 / det;
                G[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
                G[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
                G[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
                G[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
                G[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
                G[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
                for (int d = 0; d < 3; ++d)
                    for (int j = 0; j < 3; ++j) geo[(size_t)(3 * d + j) * tot + e * NP3 + n] = (float)G[d][j];
            }
            lo[e] = make_float4((float)mn[0], (float)mn[1], (float)mn[2], 0.f);
            hi[e] = make_float4((float)mx[0], (float)mx[1], (float)mx[2], 0.f);
            g[e] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    } else {
        for (int64_t e = 0; e < E; ++e) {
            const double *X = xyz + e * NP3, *Y = xyz + tot + e * NP3, *Z = xyz + 2 * tot + e * NP3;
            const double a[3] = {X[0], Y[0], Z[0]};
            const double b[3] = {X[N], Y[N * NP], Z[N * NP * NP]};
            lo[e] = make_float4((float)a[0], (float)a[1], (float)a[2], 0.f);
            hi[e] = make_float4((float)b[0], (float)b[1], (float)b[2], 0.f);
            g[e] = make_float4((float)(2.0 / (b[0] - a[0])), (float)(2.0 / (b[1] - a[1])), (float)(2.0 / (b[2] - a[2])),
                               0.f);
        }
    }
    SEM_CU(ctx, cudaSetDevice(ctx->device));
    sem_mesh *m = new sem_mesh();
    m->N = N;
    m->E = E;
    m->device = ctx->device;
    size_t bytes = sizeof(float4) * (size_t)(E > 0 ? E : 1);
    sem_status st = SEM_OK;
    do {
        if ((st = sem_cuda(ctx, cudaMalloc(&m->lo, bytes), "cudaMalloc(mesh)")) != SEM_OK) break;
        if ((st = sem_cuda(ctx, cudaMalloc(&m->hi, bytes), "cudaMalloc(mesh)")) != SEM_OK) break;
        if ((st = sem_cuda(ctx, cudaMalloc(&m->g, bytes), "cudaMalloc(mesh)")) != SEM_OK) break;
        m->owner = ctx;
        m->bytes = 3 * (int64_t)bytes;
        ctx->mem_add(m->bytes);
        if (curved) {
            m->curved = true;
            if ((st = sem_cuda(ctx, cudaMalloc(&m->geo, sizeof(float) * geo.size()), "cudaMalloc(mesh)")) != SEM_OK) break;
            m->bytes += (int64_t)(sizeof(float) * geo.size());
            ctx->mem_add((int64_t)(sizeof(float) * geo.size()));
            if ((st = sem_cuda(ctx, cudaMalloc(&m->xyzn, sizeof(float) * xyzn.size()), "cudaMalloc(mesh)")) != SEM_OK) break;
            m->bytes += (int64_t)(sizeof(float) * xyzn.size());
            ctx->mem_add((int64_t)(sizeof(float) * xyzn.size()));
            if ((st = sem_cuda(ctx, cudaMemcpy(m->geo, geo.data(), sizeof(float) * geo.size(), cudaMemcpyHostToDevice), "copy")) != SEM_OK) break;
            if ((st = sem_cuda(ctx, cudaMemcpy(m->xyzn, xyzn.data(), sizeof(float) * xyzn.size(), cudaMemcpyHostToDevice), "copy")) != SEM_OK) break;
        }
        if (E > 0) {
            if ((st = sem_cuda(ctx, cudaMemcpy(m->lo, lo.data(), sizeof(float4) * E, cudaMemcpyHostToDevice), "copy")) != SEM_OK) break;
            if ((st = sem_cuda(ctx, cudaMemcpy(m->hi, hi.data(), sizeof(float4) * E, cudaMemcpyHostToDevice), "copy")) != SEM_OK) break;
            if ((st = sem_cuda(ctx, cudaMemcpy(m->g, g.data(), sizeof(float4) * E, cudaMemcpyHostToDevice), "copy")) != SEM_OK) break;
        }
    } while (0);
    if (st != SEM_OK) {
        sem_mesh_free(m);
        return st;
    }
    *out = m;
    return SEM_OK;
}

void sem_mesh_free(sem_mesh *m)
{
    if (!m) return;
    cudaSetDevice(m->device);
    if (m->owner) m->owner->mem_add(-m->bytes);
    if (m->lo) cudaFree(m->lo);
    if (m->hi) cudaFree(m->hi);
    if (m->g) cudaFree(m->g);
    if (m->geo) cudaFree(m->geo);
    if (m->xyzn) cudaFree(m->xyzn);
    delete m;
}

sem_status sem_mesh_info(const sem_mesh *m, int *N, int64_t *E)
{
    if (!m) return SEM_ERR_ARG;
    if (N) *N = m->N;
    if (E) *E = m->E;
    return SEM_OK;
}

static sem_status check_common(sem_ctx *ctx, const sem_mesh *m, const char *fn)
{
    if (!ctx) return SEM_ERR_ARG;
    if (!m) return sem_fail(ctx, SEM_ERR_ARG, "%s: mesh is NULL", fn);
    if (m->device != ctx->device) return sem_fail(ctx, SEM_ERR_ARG, "%s: mesh lives on another device", fn);
    return sem_cuda(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
}

static sem_status check_ptr(sem_ctx *ctx, const void *p, const char *fn, const char *name, bool may_null = false,
                            unsigned align = 16)
{
    if (!p) return may_null ? SEM_OK : sem_fail(ctx, SEM_ERR_ARG, "%s: %s is NULL", fn, name);
    if ((reinterpret_cast<uintptr_t>(p) & (align - 1)) != 0)
        return sem_fail(ctx, SEM_ERR_ARG, "%s: %s is not %u-byte aligned", fn, name, align);
    return SEM_OK;
}

sem_status sem_derivatives(sem_ctx *ctx, const sem_mesh *m, const float *u, float *dudx, float *dudy, float *dudz,
                           sem_prec prec)
{
    SEM_TRY(check_common(ctx, m, "sem_derivatives"));
    if (m->E == 0) return SEM_OK;
    SEM_TRY(check_ptr(ctx, u, "sem_derivatives", "u"));
    SEM_TRY(check_ptr(ctx, dudx, "sem_derivatives", "dudx"));
    SEM_TRY(check_ptr(ctx, dudy, "sem_derivatives", "dudy"));
    SEM_TRY(check_ptr(ctx, dudz, "sem_derivatives", "dudz"));
    if (prec != SEM_FP32)
        return sem_fail(ctx, prec >= SEM_FP32 && prec <= SEM_BF16X2 ? SEM_ERR_UNSUPPORTED : SEM_ERR_ARG,
                        "sem_derivatives: precision %d not available", (int)prec);
    return deriv_launch(ctx, m, u, dudx, dudy, dudz);
}

sem_status sem_qcriterion(sem_ctx *ctx, const sem_mesh *m, const float *u, const float *v, const float *w, float *Q,
                          sem_prec prec)
{
    SEM_TRY(check_common(ctx, m, "sem_qcriterion"));
    if (m->E == 0) return SEM_OK;
    SEM_TRY(check_ptr(ctx, u, "sem_qcriterion", "u"));
    SEM_TRY(check_ptr(ctx, v, "sem_qcriterion", "v"));
    SEM_TRY(check_ptr(ctx, w, "sem_qcriterion", "w"));
    SEM_TRY(check_ptr(ctx, Q, "sem_qcriterion", "Q"));
    if (Q == u || Q == v || Q == w) return sem_fail(ctx, SEM_ERR_ARG, "sem_qcriterion: Q aliases an input");
    if (prec == SEM_FP32) return qcrit_launch(ctx, m, u, v, w, Q);
    if (prec == SEM_BF16 || prec == SEM_FP16 || prec == SEM_BF16X2 || prec == SEM_TF32) {
        if (m->curved)
            return sem_fail(ctx, SEM_ERR_UNSUPPORTED,
                            "sem_qcriterion: tensor-core precisions need axis-aligned box elements (general mesh)");
        double xi[SEM_MAX_ORDER + 1], D[(SEM_MAX_ORDER + 1) * (SEM_MAX_ORDER + 1)];
        gll_nodes(m->N, xi);
        gll_dmat(m->N, xi, D);
        return qcrit_tc_launch(ctx, m, u, v, w, Q, prec, D);
    }
    return sem_fail(ctx, SEM_ERR_ARG, "sem_qcriterion: precision %d not available", (int)prec);
}

sem_status sem_qcriterion_batch(sem_ctx *ctx, int n, const sem_mesh *const *meshes, const float *const *u,
                                const float *const *v, const float *const *w, float *const *Q)
{
    if (!ctx) return SEM_ERR_ARG;
    SEM_CU(ctx, cudaSetDevice(ctx->device));
    if (n < 0 || (n > 0 && (!meshes || !u || !v || !w || !Q)))
        return sem_fail(ctx, SEM_ERR_ARG, "sem_qcriterion_batch: bad arrays");
    for (int p = 0; p < n; ++p) {
        SEM_TRY(check_common(ctx, meshes[p], "sem_qcriterion_batch"));
        if (meshes[p]->E == 0) continue;
        SEM_TRY(check_ptr(ctx, u[p], "sem_qcriterion_batch", "u[p]"));
        SEM_TRY(check_ptr(ctx, v[p], "sem_qcriterion_batch", "v[p]"));
        SEM_TRY(check_ptr(ctx, w[p], "sem_qcriterion_batch", "w[p]"));
        SEM_TRY(check_ptr(ctx, Q[p], "sem_qcriterion_batch", "Q[p]"));
        if (Q[p] == u[p] || Q[p] == v[p] || Q[p] == w[p])
            return sem_fail(ctx, SEM_ERR_ARG, "sem_qcriterion_batch: Q[%d] aliases an input", p);
        if (meshes[p]->curved)
            return sem_fail(ctx, SEM_ERR_UNSUPPORTED,
                            "sem_qcriterion_batch: partition %d has a general (curved) mesh; use sem_qcriterion", p);
    }
    return qcrit_batch_launch(ctx, n, meshes, u, v, w, Q);
}

sem_status sem_isosurface(sem_ctx *ctx, const sem_mesh *m, const float *f, float iso, float *tris, int32_t *tri_elem,
                          int64_t cap, int64_t *ntri_out, uint8_t *cases)
{
    SEM_TRY(check_common(ctx, m, "sem_isosurface"));
    if (!ntri_out) return sem_fail(ctx, SEM_ERR_ARG, "sem_isosurface: ntri_out is NULL");
    *ntri_out = 0;
    if (cap < 0) return sem_fail(ctx, SEM_ERR_ARG, "sem_isosurface: negative cap");
    if (m->E == 0) return SEM_OK;
    SEM_TRY(check_ptr(ctx, f, "sem_isosurface", "f"));
    SEM_TRY(check_ptr(ctx, tris, "sem_isosurface", "tris", true, 4));
    SEM_TRY(check_ptr(ctx, tri_elem, "sem_isosurface", "tri_elem", true, 4));
    SEM_TRY(check_ptr(ctx, cases, "sem_isosurface", "cases", true));
    if (isnan(iso)) return sem_fail(ctx, SEM_ERR_ARG, "sem_isosurface: iso is NaN");
    return iso_run(ctx, m, f, iso, tris, tri_elem, cap, ntri_out, cases);
}

sem_status sem_isosurface_multi(sem_ctx *ctx, const sem_mesh *m, const float *f, const float *isos, int niso,
                                float *tris, int32_t *tri_elem, int64_t cap, int64_t *ntri_out, uint8_t *cases)
{
    SEM_TRY(check_common(ctx, m, "sem_isosurface_multi"));
    if (!ntri_out || !isos) return sem_fail(ctx, SEM_ERR_ARG, "sem_isosurface_multi: isos or ntri_out is NULL");
    if (niso < 1 || niso > SEM_MAX_ISO)
        return sem_fail(ctx, SEM_ERR_ARG, "sem_isosurface_multi: niso=%d outside [1,%d]", niso, SEM_MAX_ISO);
    for (int q = 0; q < niso; ++q) {
        ntri_out[q] = 0;
        if (isnan(isos[q])) return sem_fail(ctx, SEM_ERR_ARG, "sem_isosurface_multi: isovalue %d is NaN", q);
    }
    if (cap < 0) return sem_fail(ctx, SEM_ERR_ARG, "sem_isosurface_multi: negative cap");
    if (m->E == 0) return SEM_OK;
    if (m->E * (int64_t)niso > ((int64_t)1 << 31))
        return sem_fail(ctx, SEM_ERR_ARG, "sem_isosurface_multi: E*niso too large");
    SEM_TRY(check_ptr(ctx, f, "sem_isosurface_multi", "f"));
    SEM_TRY(check_ptr(ctx, tris, "sem_isosurface_multi", "tris", true, 4));
    SEM_TRY(check_ptr(ctx, tri_elem, "sem_isosurface_multi", "tri_elem", true, 4));
    SEM_TRY(check_ptr(ctx, cases, "sem_isosurface_multi", "cases", true));
    return iso_run_multi(ctx, m, f, isos, niso, tris, tri_elem, cap, ntri_out, cases);
}

sem_status sem_isosurface_multi_async(sem_ctx *ctx, const sem_mesh *m, const float *f, const float *isos, int niso,
                                      float *tris, int32_t *tri_elem, int64_t cap, int64_t *counts_dev, uint8_t *cases)
{
    SEM_TRY(check_common(ctx, m, "sem_isosurface_multi_async"));
    if (!isos || niso < 1 || niso > SEM_MAX_ISO)
        return sem_fail(ctx, SEM_ERR_ARG, "sem_isosurface_multi_async: need 1 <= niso <= %d isovalues", SEM_MAX_ISO);
    for (int q = 0; q < niso; ++q)
        if (isnan(isos[q])) return sem_fail(ctx, SEM_ERR_ARG, "sem_isosurface_multi_async: isovalue %d is NaN", q);
    if (cap < 0) return sem_fail(ctx, SEM_ERR_ARG, "sem_isosurface_multi_async: negative cap");
    SEM_TRY(check_ptr(ctx, counts_dev, "sem_isosurface_multi_async", "counts_dev", false, 8));
    if (m->E == 0) return sem_cuda(ctx, cudaMemsetAsync(counts_dev, 0, sizeof(int64_t) * (niso + 1), ctx->stream),
                                   "cudaMemsetAsync");
    if (m->E * (int64_t)niso > ((int64_t)1 << 31))
        return sem_fail(ctx, SEM_ERR_ARG, "sem_isosurface_multi_async: E*niso too large");
    SEM_TRY(check_ptr(ctx, f, "sem_isosurface_multi_async", "f"));
    SEM_TRY(check_ptr(ctx, tris, "sem_isosurface_multi_async", "tris", true, 4));
    SEM_TRY(check_ptr(ctx, tri_elem, "sem_isosurface_multi_async", "tri_elem", true, 4));
    SEM_TRY(check_ptr(ctx, cases, "sem_isosurface_multi_async", "cases", true));
    return iso_run_multi_async(ctx, m, f, isos, niso, tris, tri_elem, cap, counts_dev, cases);
}

sem_status sem_qcriterion_isosurface_async(sem_ctx *ctx, const sem_mesh *m, const float *u, const float *v,
                                           const float *w, float *Q, const float *isos, int niso, float *tris,
                                           int32_t *tri_elem, int64_t cap, int64_t *counts_dev)
{
    SEM_TRY(check_common(ctx, m, "sem_qcriterion_isosurface_async"));
    if (!isos || niso < 1 || niso > SEM_MAX_ISO)
        return sem_fail(ctx, SEM_ERR_ARG, "sem_qcriterion_isosurface_async: need 1 <= niso <= %d isovalues",
                        SEM_MAX_ISO);
    for (int q = 0; q < niso; ++q)
        if (isnan(isos[q]))
            return sem_fail(ctx, SEM_ERR_ARG, "sem_qcriterion_isosurface_async: isovalue %d is NaN", q);
    if (cap < 0) return sem_fail(ctx, SEM_ERR_ARG, "sem_qcriterion_isosurface_async: negative cap");
    SEM_TRY(check_ptr(ctx, counts_dev, "sem_qcriterion_isosurface_async", "counts_dev", false, 8));
    if (m->E == 0) return sem_cuda(ctx, cudaMemsetAsync(counts_dev, 0, sizeof(int64_t) * (niso + 1), ctx->stream),
                                   "cudaMemsetAsync");
    if (m->E * (int64_t)niso > ((int64_t)1 << 31))
        return sem_fail(ctx, SEM_ERR_ARG, "sem_qcriterion_isosurface_async: E*niso too large");
    const char *fn = "sem_qcriterion_isosurface_async";
    SEM_TRY(check_ptr(ctx, u, fn, "u"));
    SEM_TRY(check_ptr(ctx, v, fn, "v"));
    SEM_TRY(check_ptr(ctx, w, fn, "w"));
    SEM_TRY(check_ptr(ctx, Q, fn, "Q"));
    if (Q == u || Q == v || Q == w) return sem_fail(ctx, SEM_ERR_ARG, "%s: Q aliases an input", fn);
    SEM_TRY(check_ptr(ctx, tris, fn, "tris", true, 4));
    SEM_TRY(check_ptr(ctx, tri_elem, fn, "tri_elem", true, 4));
    return iso_run_q_multi_async(ctx, m, u, v, w, Q, isos, niso, tris, tri_elem, cap, counts_dev);
}

// Argument checks shared by sem_qcriterion_isosurface_fields_async and sem_frame_async;
// *total_niso receives q_niso + sum f_niso.
static sem_status check_fields_call(sem_ctx *ctx, const char *fn, const sem_mesh *m, const float *u, const float *v,
                                    const float *w, const float *Q, const float *q_isos, int q_niso, int nfields,
                                    const float *const *fields, const float *f_isos, const int *f_niso,
                                    const float *tris, const int32_t *tri_elem, int64_t cap,
                                    const int64_t *counts_dev, int *total_niso)
{
    SEM_TRY(check_common(ctx, m, fn));
    if (!q_isos || q_niso < 1 || q_niso > SEM_MAX_ISO)
        return sem_fail(ctx, SEM_ERR_ARG, "%s: need 1 <= q_niso <= %d isovalues", fn, SEM_MAX_ISO);
    if (nfields < 0 || nfields > SEM_MAX_FIELDS)
        return sem_fail(ctx, SEM_ERR_ARG, "%s: need 0 <= nfields <= %d", fn, SEM_MAX_FIELDS);
    if (nfields > 0 && (!fields || !f_isos || !f_niso))
        return sem_fail(ctx, SEM_ERR_ARG, "%s: fields, f_isos and f_niso are required when nfields > 0", fn);
    for (int q = 0; q < q_niso; ++q)
        if (isnan(q_isos[q])) return sem_fail(ctx, SEM_ERR_ARG, "%s: Q isovalue %d is NaN", fn, q);
    int tot = q_niso;
    for (int k = 0, at = 0; k < nfields; ++k) {
        if (f_niso[k] < 1 || f_niso[k] > SEM_MAX_ISO)
            return sem_fail(ctx, SEM_ERR_ARG, "%s: field %d: need 1 <= f_niso <= %d isovalues", fn, k, SEM_MAX_ISO);
        for (int q = 0; q < f_niso[k]; ++q, ++at)
            if (isnan(f_isos[at])) return sem_fail(ctx, SEM_ERR_ARG, "%s: field %d: isovalue %d is NaN", fn, k, q);
        tot += f_niso[k];
    }
    *total_niso = tot;
    if (cap < 0) return sem_fail(ctx, SEM_ERR_ARG, "%s: negative cap", fn);
    SEM_TRY(check_ptr(ctx, counts_dev, fn, "counts_dev", false, 8));
    for (int k = -1; k < nfields; ++k)
        if (m->E * (int64_t)(k < 0 ? q_niso : f_niso[k]) > ((int64_t)1 << 31))
            return sem_fail(ctx, SEM_ERR_ARG, "%s: E*niso too large", fn);
    if (m->E == 0) return SEM_OK;
    SEM_TRY(check_ptr(ctx, u, fn, "u"));
    SEM_TRY(check_ptr(ctx, v, fn, "v"));
    SEM_TRY(check_ptr(ctx, w, fn, "w"));
    SEM_TRY(check_ptr(ctx, Q, fn, "Q"));
    if (Q == u || Q == v || Q == w) return sem_fail(ctx, SEM_ERR_ARG, "%s: Q aliases an input", fn);
    for (int k = 0; k < nfields; ++k) {
        SEM_TRY(check_ptr(ctx, fields[k], fn, "fields[k]"));
        if (fields[k] == Q) return sem_fail(ctx, SEM_ERR_ARG, "%s: field %d aliases Q", fn, k);
    }
    SEM_TRY(check_ptr(ctx, tris, fn, "tris", true, 4));
    return check_ptr(ctx, tri_elem, fn, "tri_elem", true, 4);
}

sem_status sem_qcriterion_isosurface_fields_async(sem_ctx *ctx, const sem_mesh *m, const float *u, const float *v,
                                                  const float *w, float *Q, const float *q_isos, int q_niso,
                                                  int nfields, const float *const *fields, const float *f_isos,
                                                  const int *f_niso, float *tris, int32_t *tri_elem, int64_t cap,
                                                  int64_t *counts_dev)
{
    const char *fn = "sem_qcriterion_isosurface_fields_async";
    int total_niso = 0;
    SEM_TRY(check_fields_call(ctx, fn, m, u, v, w, Q, q_isos, q_niso, nfields, fields, f_isos, f_niso, tris, tri_elem,
                              cap, counts_dev, &total_niso));
    if (m->E == 0)
        return sem_cuda(ctx, cudaMemsetAsync(counts_dev, 0, sizeof(int64_t) * (total_niso + 1), ctx->stream),
                        "cudaMemsetAsync");
    return iso_run_q_fields_async(ctx, m, u, v, w, Q, q_isos, q_niso, nfields, fields, f_isos, f_niso, tris, tri_elem,
                                  cap, counts_dev);
}

static sem_status check_camera(sem_ctx *ctx, const char *fn, const sem_camera *cam, int W, int H)
{
    if (!cam) return sem_fail(ctx, SEM_ERR_ARG, "%s: cam is NULL", fn);
    if (W < 1 || H < 1 || W > 16384 || H > 16384) return sem_fail(ctx, SEM_ERR_ARG, "%s: bad size", fn);
    if (!(cam->znear > 0.f) || !(cam->zfar > cam->znear))
        return sem_fail(ctx, SEM_ERR_ARG, "%s: need 0 < znear < zfar", fn);
    if (cam->ortho ? !(cam->half_h > 0.f) : !(cam->fovy_deg > 0.f && cam->fovy_deg < 180.f))
        return sem_fail(ctx, SEM_ERR_ARG, "%s: bad projection parameters", fn);
    return SEM_OK;
}

sem_status sem_frame_async(sem_ctx *ctx, const sem_mesh *m, const float *u, const float *v, const float *w, float *Q,
                           const float *q_isos, int q_niso, int nfields, const float *const *fields,
                           const float *f_isos, const int *f_niso, float *tris, int32_t *tri_elem, int64_t cap,
                           int64_t *counts_dev, const float *seg_rgb, const sem_camera *cam, int W, int H,
                           uint8_t *rgba, float *depth)
{
    const char *fn = "sem_frame_async";
    int nseg = 0;
    SEM_TRY(check_fields_call(ctx, fn, m, u, v, w, Q, q_isos, q_niso, nfields, fields, f_isos, f_niso, tris, tri_elem,
                              cap, counts_dev, &nseg));
    SEM_TRY(check_camera(ctx, fn, cam, W, H));
    if (cap >= ((int64_t)1 << 31)) return sem_fail(ctx, SEM_ERR_ARG, "%s: cap must be below 2^31", fn);
    SEM_TRY(check_ptr(ctx, tris, fn, "tris", cap == 0, 4));
    SEM_TRY(check_ptr(ctx, rgba, fn, "rgba"));
    SEM_TRY(check_ptr(ctx, depth, fn, "depth", true));
    if (m->E == 0) {
        SEM_CU(ctx, cudaMemsetAsync(counts_dev, 0, sizeof(int64_t) * (nseg + 1), ctx->stream));
        std::vector<int64_t> zeros(nseg, 0);
        return render_run(ctx, tris, cap, zeros.data(), nseg, seg_rgb, cam, W, H, rgba, depth, counts_dev);
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    SEM_CU(ctx, cudaStreamIsCapturing(ctx->stream, &cs));
    if (nfields == 0 || (cs == cudaStreamCaptureStatusNone && !render_width_settled(ctx, W, H))) {
        // the two calls in sequence: with no further fields there is nothing for a second
        // stream to overlap, and on the first frame of this size with the autotuner on, the
        // render's launch widths are timed on a whole frame
        SEM_TRY(iso_run_q_fields_async(ctx, m, u, v, w, Q, q_isos, q_niso, nfields, fields, f_isos, f_niso, tris,
                                       tri_elem, cap, counts_dev));
        std::vector<int64_t> zeros(nseg, 0);
        return render_run(ctx, tris, cap, zeros.data(), nseg, seg_rgb, cam, W, H, rgba, depth, counts_dev);
    }
    SEM_TRY(render_frame_begin(ctx, cap, counts_dev, nseg, seg_rgb, cam, W, H, rgba, depth));
    SEM_TRY(iso_run_q_fields_async(ctx, m, u, v, w, Q, q_isos, q_niso, nfields, fields, f_isos, f_niso, tris,
                                   tri_elem, cap, counts_dev, true));
    return render_frame_end(ctx, tris);
}

sem_status sem_isosurface_multi_append_async(sem_ctx *ctx, const sem_mesh *m, const float *f, const float *isos,
                                             int niso, float *tris, int32_t *tri_elem, int64_t cap,
                                             int64_t *counts_dev, uint8_t *cases)
{
    SEM_TRY(check_common(ctx, m, "sem_isosurface_multi_append_async"));
    if (!isos || niso < 1 || niso > SEM_MAX_ISO)
        return sem_fail(ctx, SEM_ERR_ARG, "sem_isosurface_multi_append_async: need 1 <= niso <= %d isovalues",
                        SEM_MAX_ISO);
    for (int q = 0; q < niso; ++q)
        if (isnan(isos[q]))
            return sem_fail(ctx, SEM_ERR_ARG, "sem_isosurface_multi_append_async: isovalue %d is NaN", q);
    if (cap < 0) return sem_fail(ctx, SEM_ERR_ARG, "sem_isosurface_multi_append_async: negative cap");
    SEM_TRY(check_ptr(ctx, counts_dev, "sem_isosurface_multi_append_async", "counts_dev", false, 8));
    if (m->E * (int64_t)niso > ((int64_t)1 << 31))
        return sem_fail(ctx, SEM_ERR_ARG, "sem_isosurface_multi_append_async: E*niso too large");
    SEM_TRY(check_ptr(ctx, f, "sem_isosurface_multi_append_async", "f", m->E == 0));
    SEM_TRY(check_ptr(ctx, tris, "sem_isosurface_multi_append_async", "tris", true, 4));
    SEM_TRY(check_ptr(ctx, tri_elem, "sem_isosurface_multi_append_async", "tri_elem", true, 4));
    SEM_TRY(check_ptr(ctx, cases, "sem_isosurface_multi_append_async", "cases", true));
    if (m->E == 0) {
        // no triangles: every segment end equals the start
        for (int q = 1; q <= niso; ++q)
            SEM_CU(ctx, cudaMemcpyAsync(counts_dev + q, counts_dev, sizeof(int64_t), cudaMemcpyDeviceToDevice,
                                        ctx->stream));
        return SEM_OK;
    }
    return iso_run_multi_async(ctx, m, f, isos, niso, tris, tri_elem, cap, counts_dev, cases, true);
}

static sem_status render_async_checked(sem_ctx *ctx, const char *fn, const float *tris, int64_t ntri_max,
                                       const int64_t *seg_start_dev, int nseg, int max_seg, const float *seg_rgb,
                                       unsigned long long seg_mask, const sem_camera *cam, int W, int H,
                                       uint8_t *rgba, float *depth)
{
    if (!ctx) return SEM_ERR_ARG;
    SEM_CU(ctx, cudaSetDevice(ctx->device));
    SEM_TRY(check_camera(ctx, fn, cam, W, H));
    if (ntri_max < 0 || ntri_max >= ((int64_t)1 << 31) || nseg < 1 || nseg > max_seg)
        return sem_fail(ctx, SEM_ERR_ARG, "%s: bad ntri_max or nseg", fn);
    SEM_TRY(check_ptr(ctx, seg_start_dev, fn, "seg_start_dev", false, 8));
    SEM_TRY(check_ptr(ctx, tris, fn, "tris", ntri_max == 0, 4));
    SEM_TRY(check_ptr(ctx, rgba, fn, "rgba"));
    SEM_TRY(check_ptr(ctx, depth, fn, "depth", true));
    std::vector<int64_t> dummy(nseg, 0);
    return render_run(ctx, tris, ntri_max, dummy.data(), nseg, seg_rgb, cam, W, H, rgba, depth, seg_start_dev,
                      seg_mask);
}

sem_status sem_render_async(sem_ctx *ctx, const float *tris, int64_t ntri_max, const int64_t *seg_start_dev, int nseg,
                            const float *seg_rgb, const sem_camera *cam, int W, int H, uint8_t *rgba, float *depth)
{
    return render_async_checked(ctx, "sem_render_async", tris, ntri_max, seg_start_dev, nseg, 16, seg_rgb, ~0ull,
                                cam, W, H, rgba, depth);
}

sem_status sem_render_segments_async(sem_ctx *ctx, const float *tris, int64_t ntri_max, const int64_t *seg_start_dev,
                                     int nseg, const float *seg_rgb, uint64_t seg_mask, const sem_camera *cam, int W,
                                     int H, uint8_t *rgba, float *depth)
{
    return render_async_checked(ctx, "sem_render_segments_async", tris, ntri_max, seg_start_dev, nseg, 64, seg_rgb,
                                (unsigned long long)seg_mask, cam, W, H, rgba, depth);
}

sem_status sem_isosurface_noalloc(sem_ctx *ctx, const sem_mesh *m, const float *f, float iso, float *tris,
                                  int32_t *tri_elem, int64_t cap, int64_t *ntri_out, uint8_t *cases)
{
    SEM_TRY(check_common(ctx, m, "sem_isosurface_noalloc"));
    if (!ntri_out) return sem_fail(ctx, SEM_ERR_ARG, "sem_isosurface_noalloc: ntri_out is NULL");
    *ntri_out = 0;
    if (cap < 0) return sem_fail(ctx, SEM_ERR_ARG, "sem_isosurface_noalloc: negative cap");
    if (m->E > SEM_NOALLOC_MAX_ELEMENTS)
        return sem_fail(ctx, SEM_ERR_ARG,
                        "sem_isosurface_noalloc: the mesh has %lld elements, more than the %d its fixed scratch "
                        "holds; use sem_isosurface",
                        (long long)m->E, SEM_NOALLOC_MAX_ELEMENTS);
    if (m->E == 0) return SEM_OK;
    if (m->curved)
        return sem_fail(ctx, SEM_ERR_UNSUPPORTED, "sem_isosurface_noalloc: general (curved) mesh; use sem_isosurface");
    SEM_TRY(check_ptr(ctx, f, "sem_isosurface_noalloc", "f"));
    SEM_TRY(check_ptr(ctx, tris, "sem_isosurface_noalloc", "tris", true, 4));
    SEM_TRY(check_ptr(ctx, tri_elem, "sem_isosurface_noalloc", "tri_elem", true, 4));
    SEM_TRY(check_ptr(ctx, cases, "sem_isosurface_noalloc", "cases", true));
    if (isnan(iso)) return sem_fail(ctx, SEM_ERR_ARG, "sem_isosurface_noalloc: iso is NaN");
    return iso_run_noalloc(ctx, m, f, iso, tris, tri_elem, cap, ntri_out, cases);
}

sem_status sem_render(sem_ctx *ctx, const float *tris, int64_t ntri, const int64_t *seg_ntri, int nseg,
                      const float *seg_rgb, const sem_camera *cam, int W, int H, uint8_t *rgba, float *depth)
{
    if (!ctx) return SEM_ERR_ARG;
    SEM_CU(ctx, cudaSetDevice(ctx->device));
    if (!cam) return sem_fail(ctx, SEM_ERR_ARG, "sem_render: cam is NULL");
    if (W < 1 || H < 1 || W > 16384 || H > 16384) return sem_fail(ctx, SEM_ERR_ARG, "sem_render: bad size %dx%d", W, H);
    if (ntri < 0 || nseg < 1 || nseg > 16 || !seg_ntri) return sem_fail(ctx, SEM_ERR_ARG, "sem_render: bad segments");
    int64_t sum = 0;
    for (int s = 0; s < nseg; ++s) {
        if (seg_ntri[s] < 0) return sem_fail(ctx, SEM_ERR_ARG, "sem_render: negative segment size");
        sum += seg_ntri[s];
    }
    if (sum != ntri) return sem_fail(ctx, SEM_ERR_ARG, "sem_render: segments sum to %lld, ntri=%lld", (long long)sum, (long long)ntri);
    if (ntri >= ((int64_t)1 << 31)) return sem_fail(ctx, SEM_ERR_ARG, "sem_render: ntri >= 2^31");
    SEM_TRY(check_ptr(ctx, tris, "sem_render", "tris", ntri == 0, 4));
    SEM_TRY(check_ptr(ctx, rgba, "sem_render", "rgba"));
    SEM_TRY(check_ptr(ctx, depth, "sem_render", "depth", true));
    if (!(cam->znear > 0.f) || !(cam->zfar > cam->znear))
        return sem_fail(ctx, SEM_ERR_ARG, "sem_render: need 0 < znear < zfar");
    if (cam->ortho ? !(cam->half_h > 0.f) : !(cam->fovy_deg > 0.f && cam->fovy_deg < 180.f))
        return sem_fail(ctx, SEM_ERR_ARG, "sem_render: bad projection parameters");
    return render_run(ctx, tris, ntri, seg_ntri, nseg, seg_rgb, cam, W, H, rgba, depth);
}

sem_status sem_surface_measures(sem_ctx *ctx, const float *tris, int64_t ntri, double *out_host)
{
    if (!ctx) return SEM_ERR_ARG;
    SEM_CU(ctx, cudaSetDevice(ctx->device));
    if (!out_host || ntri < 0) return sem_fail(ctx, SEM_ERR_ARG, "sem_surface_measures: bad arguments");
    out_host[0] = out_host[1] = 0.0;
    if (ntri == 0) return SEM_OK;
    SEM_TRY(check_ptr(ctx, tris, "sem_surface_measures", "tris", false, 4));
    return measures_run(ctx, tris, ntri, out_host);
}

sem_status sem_field_max(sem_ctx *ctx, const float *f, int64_t n, float *max_host)
{
    if (!ctx) return SEM_ERR_ARG;
    SEM_CU(ctx, cudaSetDevice(ctx->device));
    if (!max_host || n < 1) return sem_fail(ctx, SEM_ERR_ARG, "sem_field_max: bad arguments");
    SEM_TRY(check_ptr(ctx, f, "sem_field_max", "f"));
    return fieldmax_run(ctx, f, n, max_host);
}

}  // extern "C"
