// sem_scan.cu -- device-wide exclusive scan (counts -> offsets) and the global reductions
// behind the checks: FP64 surface area / enclosed volume and the field maximum.
#include <cuda_runtime.h>
#include <math.h>

#include "sem_internal.cuh"

#define SCAN_THREADS 1024
#define SCAN_ITEMS 4
#define SCAN_TILE (SCAN_THREADS * SCAN_ITEMS)

size_t scan_tmp_bytes(int64_t n)
{
    const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    return ((sizeof(int64_t) * (size_t)(nb + 1) + 255) / 256) * 256;
}

size_t scan_live_tmp_bytes(int64_t n)
{
    const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    return ((sizeof(int64_t) * (size_t)(2 * nb + 1) + 255) / 256) * 256;
}

// block-wide exclusive scan of one int64 per thread; returns the block total in *total
__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t *s_warp, int64_t &total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int64_t incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
    }
    if (lane == 31) s_warp[w] = incl;
    __syncthreads();
    if (w == 0) {
        int64_t x = lane < nw ? s_warp[lane] : 0;
        int64_t xi = x;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, xi, d);
            if (lane >= d) xi += y;
        }
        if (lane < nw) s_warp[lane] = xi - x;  // exclusive warp offsets
        if (lane == 31) s_warp[32] = xi;
    }
    __syncthreads();
    const int64_t r = s_warp[w] + incl - v;
    total = s_warp[32];
    __syncthreads();
    return r;
}

// block-wide exclusive scan of two int64 per thread at once (a, b); totals in ta, tb
__device__ __forceinline__ void block_excl_scan2(int64_t a, int64_t b, int64_t (*s_warp)[33], int64_t &ea,
                                                 int64_t &eb, int64_t &ta, int64_t &tb)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int64_t ia = a, ib = b;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int64_t ya = __shfl_up_sync(0xffffffffu, ia, d), yb = __shfl_up_sync(0xffffffffu, ib, d);
        if (lane >= d) {
            ia += ya;
            ib += yb;
        }
    }
    if (lane == 31) {
        s_warp[0][w] = ia;
        s_warp[1][w] = ib;
    }
    __syncthreads();
    if (w < 2) {
        const int64_t x = lane < nw ? s_warp[w][lane] : 0;
        int64_t xi = x;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, xi, d);
            if (lane >= d) xi += y;
        }
        if (lane < nw) s_warp[w][lane] = xi - x;
        if (lane == 31) s_warp[w][32] = xi;
    }
    __syncthreads();
    ea = s_warp[0][w] + ia - a;
    eb = s_warp[1][w] + ib - b;
    ta = s_warp[0][32];
    tb = s_warp[1][32];
    __syncthreads();
}

// Single-pass scan with decoupled look-back (Merrill & Garland, "Single-pass Parallel Prefix
// Scan with Decoupled Look-back", NVIDIA technical report, 2016).  Each block takes the next
// tile from a ticket counter, scans it, publishes the tile's sum, then folds the published
// values of the tiles before it -- tile sums until it meets a published inclusive prefix -- and
// publishes its own inclusive prefix.  Tiles are taken in ticket order, so a block waits only
// on tiles held by blocks that are already running and never wait on it: every wait ends.  Each
// is bounded all the same (SEM_WAIT_LIMIT polls, then SEM_ERR_TIMEOUT on the device flag).
// state[0] is the ticket, state[1 + t] tile t's status: 2 flag bits (0 nothing yet, 1 the tile
// sum, 2 the inclusive prefix) above a 62-bit value; the caller zeroes state before the launch.
#define LB_SHIFT 62
#define LB_VALUE ((1ull << LB_SHIFT) - 1ull)

__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// One warp's look-back over the status words st[0 .. tile]: publishes the tile's sum `tot`,
// folds the published values of the tiles before it and publishes the tile's inclusive prefix;
// returns the sum of all tiles before it (on every lane).
__device__ __forceinline__ int64_t lookback_warp(unsigned long long *st, int64_t tile, int64_t tot, int *err, int lane)
{
    if (lane == 0) st_release_u64(st + tile, ((tile == 0 ? 2ull : 1ull) << LB_SHIFT) | (unsigned long long)tot);
    int64_t before = 0;
    int64_t p = tile - 1;  // the nearest tile not folded in yet
    long long polls = 0;
    while (p >= 0) {
        // lane l reads tile p - l; before tile 0 there is an inclusive prefix of 0
        const int64_t q = p - lane;
        const unsigned long long w = q >= 0 ? ld_acquire_u64(st + q) : (2ull << LB_SHIFT);
        const unsigned flag = (unsigned)(w >> LB_SHIFT);
        const unsigned nr = __ballot_sync(0xffffffffu, flag == 0u);
        const unsigned pm = __ballot_sync(0xffffffffu, flag == 2u);
        const int kp = pm ? __ffs(pm) - 1 : 32;  // nearest lane holding an inclusive prefix
        const int kn = nr ? __ffs(nr) - 1 : 32;  // nearest lane whose tile has published nothing
        const int take = min(kp + 1, kn);        // lanes [0, take): tile sums (and the prefix)
        int64_t part = lane < take ? (int64_t)(w & LB_VALUE) : 0;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) part += __shfl_xor_sync(0xffffffffu, part, d);
        before += part;
        if (kp < kn) break;  // reached an inclusive prefix
        p -= take;
        if (take == 0 && ++polls >= SEM_WAIT_LIMIT) {
            if (lane == 0) atomicOr(err, 1 << SEM_ERR_TIMEOUT);
            break;
        }
    }
    if (lane == 0 && tile > 0) st_release_u64(st + tile, (2ull << LB_SHIFT) | (unsigned long long)(before + tot));
    return before;
}

// With LIVE, the same pass also lists the entries with a positive value: live[0 .. nlive) are
// their indices in increasing order and *nlive their number.  That second prefix (of the flags
// [in > 0]) has its own status words, state[1 + nb + t], and its own look-back, run by warp 1
// while warp 0 runs the first.
template <bool LIVE>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_lookback(const int32_t *__restrict__ in, int64_t n, int64_t nb,
                                                                int64_t *__restrict__ out,
                                                                unsigned long long *__restrict__ state, int *err,
                                                                int64_t *__restrict__ live,
                                                                unsigned long long *__restrict__ nlive)
{
    __shared__ int64_t s_w[2][33];
    __shared__ int64_t s_tile, s_before, s_lbefore;
    if (threadIdx.x == 0) s_tile = (int64_t)atomicAdd(state, 1ull);
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t base = tile * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    int64_t x[SCAN_ITEMS];
    if (base + SCAN_ITEMS <= n) {
        const int4 c = *reinterpret_cast<const int4 *>(in + base);  // in is 16-byte aligned
        x[0] = c.x;
        x[1] = c.y;
        x[2] = c.z;
        x[3] = c.w;
    } else {
#pragma unroll
        for (int q = 0; q < SCAN_ITEMS; ++q) x[q] = base + q < n ? in[base + q] : 0;
    }
    int64_t v = 0, lv = 0;
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        v += x[q];
        lv += x[q] > 0 ? 1 : 0;
    }
    int64_t ex, tot, lex = 0, ltot = 0;
    if constexpr (LIVE) block_excl_scan2(v, lv, s_w, ex, lex, tot, ltot);
    else ex = block_excl_scan(v, s_w[0], tot);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w == 0) {
        const int64_t before = lookback_warp(state + 1, tile, tot, err, lane);
        if (lane == 0) s_before = before;
    } else if (LIVE && w == 1) {
        const int64_t lbefore = lookback_warp(state + 1 + nb, tile, ltot, err, lane);
        if (lane == 0) s_lbefore = lbefore;
    }
    __syncthreads();
    int64_t run = s_before + ex;
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        if (base + q < n) out[base + q] = run;
        run += x[q];
    }
    if constexpr (LIVE) {
        int64_t at = s_lbefore + lex;
#pragma unroll
        for (int q = 0; q < SCAN_ITEMS; ++q)
            if (x[q] > 0) live[at++] = base + q;
        if (tile == nb - 1 && threadIdx.x == 0) *nlive = (unsigned long long)(s_lbefore + ltot);
    }
    if (tile == nb - 1 && threadIdx.x == 0) out[n] = s_before + tot;
}

// One block for small inputs: thread t scans its contiguous chunk of ceil(n / 1024) entries
// (sum, block-wide scan of the sums, then the chunk's offsets), so the whole scan is a single
// launch with no state to reset; used up to SCAN_SINGLE_MAX entries (8 per thread: beyond that
// one SM's serial chunks cost more than a multi-block scan, measured 194 us against 20 us at
// 98304 entries).
#define SCAN_SINGLE_MAX (SCAN_THREADS * 8)
template <bool LIVE>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_single(const int32_t *__restrict__ in, int64_t n,
                                                              int64_t *__restrict__ out, int64_t *__restrict__ live,
                                                              unsigned long long *__restrict__ nlive)
{
    __shared__ int64_t s_w[2][33];
    const int64_t per = (n + SCAN_THREADS - 1) / SCAN_THREADS;
    const int64_t lo = min(n, (int64_t)threadIdx.x * per), hi = min(n, lo + per);
    int64_t v = 0, lv = 0;
    for (int64_t i = lo; i < hi; ++i) {
        const int32_t c = in[i];
        v += c;
        lv += c > 0 ? 1 : 0;
    }
    int64_t run, tot, lrun = 0, ltot = 0;
    if constexpr (LIVE) block_excl_scan2(v, lv, s_w, run, lrun, tot, ltot);
    else run = block_excl_scan(v, s_w[0], tot);
    for (int64_t i = lo; i < hi; ++i) {
        const int32_t c = in[i];
        out[i] = run;
        run += c;
        if (LIVE && c > 0) live[lrun++] = i;
    }
    if (threadIdx.x == 0) {
        out[n] = tot;
        if constexpr (LIVE) *nlive = (unsigned long long)ltot;
    }
}

template <bool LIVE>
static sem_status scan_run(sem_ctx *ctx, const int32_t *in, int64_t *out, int64_t n, void *tmp, int64_t *live,
                           unsigned long long *nlive)
{
    if (n <= 0) {
        SEM_CU(ctx, cudaMemsetAsync(out, 0, sizeof(int64_t), ctx->stream));
        if (LIVE) SEM_CU(ctx, cudaMemsetAsync(nlive, 0, sizeof(unsigned long long), ctx->stream));
        return SEM_OK;
    }
    if (n <= SCAN_SINGLE_MAX) {
        SEM_TRACED(ctx, "k_scan_single",
                   k_scan_single<LIVE><<<1, SCAN_THREADS, 0, ctx->stream>>>(in, n, out, live, nlive));
        return sem_cuda(ctx, cudaGetLastError(), "scan launch");
    }
    if ((reinterpret_cast<uintptr_t>(in) & 15u) != 0)
        return sem_fail(ctx, SEM_ERR_ARG, "scan: counts not 16-byte aligned");
    const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    auto *state = reinterpret_cast<unsigned long long *>(tmp);
    const size_t words = (size_t)(LIVE ? 2 * nb + 1 : nb + 1);
    SEM_CU(ctx, cudaMemsetAsync(state, 0, sizeof(unsigned long long) * words, ctx->stream));
    SEM_TRACED(ctx, "k_scan_lookback", k_scan_lookback<LIVE><<<(unsigned)nb, SCAN_THREADS, 0, ctx->stream>>>(
        in, n, nb, out, state, ctx->d_flag, live, nlive));
    return sem_cuda(ctx, cudaGetLastError(), "scan launch");
}

sem_status scan_i32_i64(sem_ctx *ctx, const int32_t *in, int64_t *out, int64_t n, void *tmp)
{
    return scan_run<false>(ctx, in, out, n, tmp, nullptr, nullptr);
}

sem_status scan_i32_i64_live(sem_ctx *ctx, const int32_t *in, int64_t *out, int64_t n, void *tmp, int64_t *live,
                             unsigned long long *nlive)
{
    return scan_run<true>(ctx, in, out, n, tmp, live, nlive);
}

sem_status scan_load_kernels(sem_ctx *ctx)
{
    cudaFuncAttributes a;
    SEM_CU(ctx, cudaFuncGetAttributes(&a, k_scan_single<false>));
    SEM_CU(ctx, cudaFuncGetAttributes(&a, k_scan_lookback<false>));
    return SEM_OK;
}

// ------------------------------------------------------------------------------------------
// FP64 surface area and divergence-theorem volume: area = sum |(p1-p0)x(p2-p0)|/2,
// volume = sum p0.(p1 x p2)/6.
__global__ void k_measures(const float *__restrict__ tris, int64_t ntri, double *__restrict__ acc)
{
    double a = 0.0, v = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ntri; t += (int64_t)gridDim.x * blockDim.x) {
        const float *p = tris + t * 9;
        double P[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) P[q] = (double)p[q];
        const double ax = P[3] - P[0], ay = P[4] - P[1], az = P[5] - P[2];
        const double bx = P[6] - P[0], by = P[7] - P[1], bz = P[8] - P[2];
        const double nx = ay * bz - az * by, ny = az * bx - ax * bz, nz = ax * by - ay * bx;
        a += 0.5 * sqrt(nx * nx + ny * ny + nz * nz);
        const double cx = P[4] * P[8] - P[5] * P[7], cy = P[5] * P[6] - P[3] * P[8], cz = P[3] * P[7] - P[4] * P[6];
        v += (P[0] * cx + P[1] * cy + P[2] * cz) / 6.0;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, d);
        v += __shfl_xor_sync(0xffffffffu, v, d);
    }
    __shared__ double s[2][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        s[0][w] = a;
        s[1][w] = v;
    }
    __syncthreads();
    if (w == 0) {
        a = lane < (int)(blockDim.x >> 5) ? s[0][lane] : 0.0;
        v = lane < (int)(blockDim.x >> 5) ? s[1][lane] : 0.0;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, d);
            v += __shfl_xor_sync(0xffffffffu, v, d);
        }
        if (lane == 0) {
            atomicAdd(acc, a);
            atomicAdd(acc + 1, v);
        }
    }
}

sem_status measures_run(sem_ctx *ctx, const float *tris, int64_t ntri, double *out_host)
{
    void *scr;
    SEM_TRY(sem_scratch(ctx, SCR_MISC, 256, &scr));
    double *acc = reinterpret_cast<double *>(scr);
    SEM_CU(ctx, cudaMemsetAsync(acc, 0, 2 * sizeof(double), ctx->stream));
    int64_t grid = (ntri + 255) / 256;
    if (grid > 8 * ctx->sm_count) grid = 8 * ctx->sm_count;
    SEM_TRACED(ctx, "k_measures", k_measures<<<(unsigned)grid, 256, 0, ctx->stream>>>(tris, ntri, acc));
    SEM_CU(ctx, cudaGetLastError());
    SEM_CU(ctx, cudaMemcpyAsync(ctx->h_pinned_d, acc, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    SEM_CU(ctx, cudaStreamSynchronize(ctx->stream));
    out_host[0] = ctx->h_pinned_d[0];
    out_host[1] = ctx->h_pinned_d[1];
    return SEM_OK;
}

// ------------------------------------------------------------------------------------------
// Field maximum: floats mapped to order-preserving unsigned keys, atomicMax on the key.
__device__ __forceinline__ unsigned fkey(float f)
{
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__global__ void k_fieldmax(const float *__restrict__ f, int64_t n, unsigned *__restrict__ out)
{
    unsigned best = 0u;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = f[i];
        if (!isnan(v)) best = max(best, fkey(v));
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, d));
    if ((threadIdx.x & 31) == 0) atomicMax(out, best);
}

sem_status fieldmax_run(sem_ctx *ctx, const float *f, int64_t n, float *out_host)
{
    void *scr;
    SEM_TRY(sem_scratch(ctx, SCR_MISC, 256, &scr));
    unsigned *key = reinterpret_cast<unsigned *>(scr);
    SEM_CU(ctx, cudaMemsetAsync(key, 0, sizeof(unsigned), ctx->stream));
    int64_t grid = (n + 255) / 256;
    if (grid > 8 * ctx->sm_count) grid = 8 * ctx->sm_count;
    SEM_TRACED(ctx, "k_fieldmax", k_fieldmax<<<(unsigned)grid, 256, 0, ctx->stream>>>(f, n, key));
    SEM_CU(ctx, cudaGetLastError());
    SEM_CU(ctx, cudaMemcpyAsync(ctx->h_pinned, key, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
    SEM_CU(ctx, cudaStreamSynchronize(ctx->stream));
    unsigned k;
    memcpy(&k, ctx->h_pinned, sizeof k);
    if (k == 0u) {
        *out_host = NAN;
        return SEM_OK;
    }
    const unsigned u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    float r;
    memcpy(&r, &u, sizeof r);
    *out_host = r;
    return SEM_OK;
}
