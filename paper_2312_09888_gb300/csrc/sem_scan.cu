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

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const int32_t *__restrict__ in, int64_t n,
                                                              int64_t *__restrict__ bsum)
{
    __shared__ int64_t s_w[33];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    int64_t v = 0;
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q)
        if (base + q < n) v += in[base + q];
    int64_t tot;
    block_excl_scan(v, s_w, tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// single block: exclusive scan of the nb block sums in place; bsum[nb] = grand total
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_blocks(int64_t *__restrict__ bsum, int64_t nb)
{
    __shared__ int64_t s_w[33];
    int64_t carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += SCAN_THREADS) {
        const int64_t b = b0 + threadIdx.x;
        const int64_t v = b < nb ? bsum[b] : 0;
        int64_t tot;
        const int64_t ex = block_excl_scan(v, s_w, tot);
        if (b < nb) bsum[b] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) bsum[nb] = carry;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_apply(const int32_t *__restrict__ in, int64_t n,
                                                             const int64_t *__restrict__ bsum, int64_t nb,
                                                             int64_t *__restrict__ out)
{
    __shared__ int64_t s_w[33];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    int64_t x[SCAN_ITEMS];
    int64_t v = 0;
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        x[q] = base + q < n ? in[base + q] : 0;
        v += x[q];
    }
    int64_t tot;
    int64_t run = block_excl_scan(v, s_w, tot) + bsum[blockIdx.x];
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        if (base + q < n) out[base + q] = run;
        run += x[q];
    }
    if (blockIdx.x == nb - 1 && threadIdx.x == 0) out[n] = bsum[nb];
}

// One launch for up to SCAN_SELF_MAX_TILES tiles: block b sums the counts of the tiles before
// its own by itself (16-byte loads of at most (SCAN_SELF_MAX_TILES - 1) * 16 KB, just written by
// the producer and still in L2), then scans its tile -- no tile-sum pass, no inter-block wait.
#define SCAN_SELF_MAX_TILES 32
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_self(const int32_t *__restrict__ in, int64_t n, int64_t nb,
                                                            int64_t *__restrict__ out)
{
    __shared__ int64_t s_w[33];
    // counts before this tile: b * SCAN_TILE of them, a multiple of 4 (in is 16-byte aligned)
    const int4 *in4 = reinterpret_cast<const int4 *>(in);
    // (SCAN_TILE / 4) / SCAN_THREADS = 1 vector per thread and tile: eight tiles' loads in flight
    static_assert(SCAN_TILE / 4 == SCAN_THREADS, "one 16-byte load per thread and tile");
    int64_t pre = 0;
    const int nbefore = (int)blockIdx.x;
    for (int t0 = 0; t0 < nbefore; t0 += 8) {
        int4 c[8];
#pragma unroll
        for (int k = 0; k < 8; ++k)
            c[k] = t0 + k < nbefore ? in4[(int64_t)(t0 + k) * SCAN_THREADS + threadIdx.x] : make_int4(0, 0, 0, 0);
#pragma unroll
        for (int k = 0; k < 8; ++k) pre += (int64_t)c[k].x + c[k].y + c[k].z + c[k].w;
    }
    int64_t before;
    block_excl_scan(pre, s_w, before);
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    int64_t x[SCAN_ITEMS];
    int64_t v = 0;
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        x[q] = base + q < n ? in[base + q] : 0;
        v += x[q];
    }
    int64_t tot;
    int64_t run = block_excl_scan(v, s_w, tot) + before;
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        if (base + q < n) out[base + q] = run;
        run += x[q];
    }
    if (blockIdx.x == nb - 1 && threadIdx.x == 0) out[n] = before + tot;
}

// One block for small inputs: thread t scans its contiguous chunk of ceil(n / 1024) entries
// (sum, block-wide scan of the sums, then the chunk's offsets), so the whole scan is a single
// launch; used up to SCAN_SINGLE_MAX entries (8 per thread: beyond that one SM's serial chunks
// cost more than the three-kernel scan, measured 194 us against 20 us at 98304 entries).
#define SCAN_SINGLE_MAX (SCAN_THREADS * 8)
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_single(const int32_t *__restrict__ in, int64_t n,
                                                              int64_t *__restrict__ out)
{
    __shared__ int64_t s_w[33];
    const int64_t per = (n + SCAN_THREADS - 1) / SCAN_THREADS;
    const int64_t lo = min(n, (int64_t)threadIdx.x * per), hi = min(n, lo + per);
    int64_t v = 0;
    for (int64_t i = lo; i < hi; ++i) v += in[i];
    int64_t tot;
    int64_t run = block_excl_scan(v, s_w, tot);
    for (int64_t i = lo; i < hi; ++i) {
        out[i] = run;
        run += in[i];
    }
    if (threadIdx.x == 0) out[n] = tot;
}

sem_status scan_i32_i64(sem_ctx *ctx, const int32_t *in, int64_t *out, int64_t n, void *tmp)
{
    if (n <= 0) {
        SEM_CU(ctx, cudaMemsetAsync(out, 0, sizeof(int64_t), ctx->stream));
        return SEM_OK;
    }
    if (n <= SCAN_SINGLE_MAX) {
        SEM_TRACED(ctx, "k_scan_single", k_scan_single<<<1, SCAN_THREADS, 0, ctx->stream>>>(in, n, out));
        return sem_cuda(ctx, cudaGetLastError(), "scan launch");
    }
    const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb <= SCAN_SELF_MAX_TILES && (reinterpret_cast<uintptr_t>(in) & 15u) == 0) {
        SEM_TRACED(ctx, "k_scan_self", k_scan_self<<<(unsigned)nb, SCAN_THREADS, 0, ctx->stream>>>(in, n, nb, out));
        return sem_cuda(ctx, cudaGetLastError(), "scan launch");
    }
    int64_t *bsum = reinterpret_cast<int64_t *>(tmp);
    SEM_TRACED(ctx, "k_scan_reduce", k_scan_reduce<<<(unsigned)nb, SCAN_THREADS, 0, ctx->stream>>>(in, n, bsum));
    SEM_TRACED(ctx, "k_scan_blocks", k_scan_blocks<<<1, SCAN_THREADS, 0, ctx->stream>>>(bsum, nb));
    SEM_TRACED(ctx, "k_scan_apply", k_scan_apply<<<(unsigned)nb, SCAN_THREADS, 0, ctx->stream>>>(in, n, bsum, nb, out));
    return sem_cuda(ctx, cudaGetLastError(), "scan launch");
}

sem_status scan_load_kernels(sem_ctx *ctx)
{
    cudaFuncAttributes a;
    SEM_CU(ctx, cudaFuncGetAttributes(&a, k_scan_single));
    SEM_CU(ctx, cudaFuncGetAttributes(&a, k_scan_self));
    SEM_CU(ctx, cudaFuncGetAttributes(&a, k_scan_reduce));
    SEM_CU(ctx, cudaFuncGetAttributes(&a, k_scan_blocks));
    SEM_CU(ctx, cudaFuncGetAttributes(&a, k_scan_apply));
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
