// sem_render.cu -- tiled z-buffer rasteriser into a headless RGBA8 + depth image.
//
// Conventions (same statement as the header): pixel centres (x+.5, y+.5), edge functions with
// the top-left fill rule on the triangle made clockwise on screen (y down), zero-area and
// near/far-crossing triangles dropped, depth interpolated in screen space, smallest
// (depth, triangle index) wins, flat headlight shading c = rgb (0.15 + 0.85 |n.l|).
//
// Passes:
//   k_setup   one thread per triangle: project, normalise winding, write a 48-byte setup
//             record, count the 16x16-pixel tiles its (one-pixel-widened) bounding box
//             touches (atomicAdd per tile);
//   scan      tile counts -> tile list offsets (read back once to size the lists);
//   k_bin     one thread per triangle: append its index to every touched tile's list;
//   k_raster  one CTA per tile: a shared-memory key buffer of 64-bit (depth bits << 32 | id),
//             resolved with shared-memory atomicMin, so the result is independent of the order
//             the triangles are processed in; then each thread shades its pixel.
#include <cuda_runtime.h>
#include <math.h>

#include "sem_internal.cuh"

#define TILE 16
#define RT_THREADS (TILE * TILE)

struct RenderParams {
    float eye[3], s[3], u[3], f[3];
    float ax, ay;        // projection scales
    float znear, zfar;   // clip range on z_view
    float za, zb;        // depth: ortho (zv - znear)*za ; perspective zb*(1 - znear/zv)
    int ortho;
    int W, H, TW, TH;
    int nseg;
    int seg_end[16];
    float rgb[16][3];
};

// 48-byte setup record: screen x/y of the three (clockwise) vertices, depths, area and the
// widened pixel box.  valid == 0 marks a dropped triangle.
struct __align__(16) TriSetup {
    float x0, y0, x1, y1;
    float x2, y2, z0, z1;
    float z2, area;
    short px0, py0, px1, py1;
};

__device__ __forceinline__ bool top_left(float ax, float ay, float bx, float by)
{
    const float dx = bx - ax, dy = by - ay;
    return (dy < 0.f) || (dy == 0.f && dx > 0.f);
}

__device__ __forceinline__ bool project(const RenderParams &P, const float *p, float &sx, float &sy, float &sz)
{
    const float dx = p[0] - P.eye[0], dy = p[1] - P.eye[1], dz = p[2] - P.eye[2];
    const float xv = P.s[0] * dx + P.s[1] * dy + P.s[2] * dz;
    const float yv = P.u[0] * dx + P.u[1] * dy + P.u[2] * dz;
    const float zv = P.f[0] * dx + P.f[1] * dy + P.f[2] * dz;
    if (!(zv > P.znear && zv < P.zfar)) return false;
    float xn, yn;
    if (P.ortho) {
        xn = xv * P.ax;
        yn = yv * P.ay;
        sz = (zv - P.znear) * P.za;
    } else {
        xn = xv / zv * P.ax;
        yn = yv / zv * P.ay;
        sz = P.zb * (1.f - P.znear / zv);
    }
    sx = (xn + 1.f) * 0.5f * (float)P.W;
    sy = (1.f - yn) * 0.5f * (float)P.H;
    return true;
}

__global__ void k_setup(const float *__restrict__ tris, int ntri, const __grid_constant__ RenderParams P,
                        TriSetup *__restrict__ rec, int32_t *__restrict__ tile_cnt)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntri) return;
    const float *p = tris + (int64_t)t * 9;
    TriSetup r;
    r.px0 = 1;
    r.px1 = 0;  // empty box unless valid
    r.py0 = 1;
    r.py1 = 0;
    float x[3], y[3], z[3];
    bool ok = project(P, p, x[0], y[0], z[0]) && project(P, p + 3, x[1], y[1], z[1]) &&
              project(P, p + 6, x[2], y[2], z[2]);
    float area = 0.f;
    if (ok) {
        area = (x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0]);
        if (!(area != 0.f) || isnan(area)) ok = false;
    }
    if (ok && area < 0.f) {
        float tx = x[1], ty = y[1], tz = z[1];
        x[1] = x[2]; y[1] = y[2]; z[1] = z[2];
        x[2] = tx; y[2] = ty; z[2] = tz;
        area = -area;
    }
    if (ok) {
        const float mnx = fminf(x[0], fminf(x[1], x[2])), mxx = fmaxf(x[0], fmaxf(x[1], x[2]));
        const float mny = fminf(y[0], fminf(y[1], y[2])), mxy = fmaxf(y[0], fmaxf(y[1], y[2]));
        // candidate pixels: centre box widened by one pixel; the edge functions decide
        const float fx0 = fmaxf(0.f, floorf(mnx) - 1.f), fx1 = fminf((float)(P.W - 1), ceilf(mxx) + 1.f);
        const float fy0 = fmaxf(0.f, floorf(mny) - 1.f), fy1 = fminf((float)(P.H - 1), ceilf(mxy) + 1.f);
        if (fx0 <= fx1 && fy0 <= fy1) {
            r.px0 = (short)fx0;
            r.px1 = (short)fx1;
            r.py0 = (short)fy0;
            r.py1 = (short)fy1;
        }
    }
    r.x0 = x[0]; r.y0 = y[0]; r.x1 = x[1]; r.y1 = y[1];
    r.x2 = x[2]; r.y2 = y[2]; r.z0 = z[0]; r.z1 = z[1];
    r.z2 = z[2]; r.area = area;
    rec[t] = r;
    if (r.px0 <= r.px1 && r.py0 <= r.py1) {
        for (int ty = r.py0 / TILE; ty <= r.py1 / TILE; ++ty)
            for (int tx = r.px0 / TILE; tx <= r.px1 / TILE; ++tx) atomicAdd(&tile_cnt[ty * P.TW + tx], 1);
    }
}

__global__ void k_bin(const TriSetup *__restrict__ rec, int ntri, int TW, const int64_t *__restrict__ tile_off,
                      int32_t *__restrict__ tile_cur, int32_t *__restrict__ list)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntri) return;
    const TriSetup r = rec[t];
    if (!(r.px0 <= r.px1 && r.py0 <= r.py1)) return;
    for (int ty = r.py0 / TILE; ty <= r.py1 / TILE; ++ty)
        for (int tx = r.px0 / TILE; tx <= r.px1 / TILE; ++tx) {
            const int tile = ty * TW + tx;
            const int pos = atomicAdd(&tile_cur[tile], 1);
            list[tile_off[tile] + pos] = t;
        }
}

__global__ void __launch_bounds__(RT_THREADS) k_raster(const float *__restrict__ tris, const TriSetup *__restrict__ rec,
                                                       const int64_t *__restrict__ tile_off,
                                                       const int32_t *__restrict__ list,
                                                       const __grid_constant__ RenderParams P, uchar4 *__restrict__ rgba,
                                                       float *__restrict__ depth)
{
    __shared__ unsigned long long keys[RT_THREADS];
    const int tile = blockIdx.x;
    const int tx = tile % P.TW, ty = tile / P.TW;
    const int X0 = tx * TILE, Y0 = ty * TILE;
    keys[threadIdx.x] = ~0ull;
    __syncthreads();
    const int64_t beg = tile_off[tile], end = tile_off[tile + 1];
    for (int64_t q = beg + threadIdx.x; q < end; q += RT_THREADS) {
        const int t = list[q];
        const TriSetup r = rec[t];
        const int px0 = max((int)r.px0, X0), px1 = min((int)r.px1, X0 + TILE - 1);
        const int py0 = max((int)r.py0, Y0), py1 = min((int)r.py1, Y0 + TILE - 1);
        const bool tl0 = top_left(r.x0, r.y0, r.x1, r.y1);
        const bool tl1 = top_left(r.x1, r.y1, r.x2, r.y2);
        const bool tl2 = top_left(r.x2, r.y2, r.x0, r.y0);
        const float inv = 1.f / r.area;
        for (int py = py0; py <= py1; ++py) {
            const float cy = (float)py + 0.5f;
            for (int px = px0; px <= px1; ++px) {
                const float cx = (float)px + 0.5f;
                const float e0 = (r.x1 - r.x0) * (cy - r.y0) - (r.y1 - r.y0) * (cx - r.x0);
                const float e1 = (r.x2 - r.x1) * (cy - r.y1) - (r.y2 - r.y1) * (cx - r.x1);
                const float e2 = (r.x0 - r.x2) * (cy - r.y2) - (r.y0 - r.y2) * (cx - r.x2);
                const bool in = (e0 > 0.f || (e0 == 0.f && tl0)) && (e1 > 0.f || (e1 == 0.f && tl1)) &&
                                (e2 > 0.f || (e2 == 0.f && tl2));
                if (!in) continue;
                float z = (e1 * r.z0 + e2 * r.z1 + e0 * r.z2) * inv;
                z = fminf(fmaxf(z, 0.f), 1.f);
                const unsigned long long key = ((unsigned long long)__float_as_uint(z) << 32) | (unsigned)t;
                atomicMin(&keys[(py - Y0) * TILE + (px - X0)], key);
            }
        }
    }
    __syncthreads();
    const int px = X0 + (threadIdx.x % TILE), py = Y0 + (threadIdx.x / TILE);
    if (px >= P.W || py >= P.H) return;
    const unsigned long long key = keys[threadIdx.x];
    const int64_t pix = (int64_t)py * P.W + px;
    if (key == ~0ull) {
        rgba[pix] = make_uchar4(0, 0, 0, 0);
        if (depth) depth[pix] = 1.f;
        return;
    }
    const int t = (int)(key & 0xffffffffu);
    const float *p = tris + (int64_t)t * 9;
    const float ax = p[3] - p[0], ay = p[4] - p[1], az = p[5] - p[2];
    const float bx = p[6] - p[0], by = p[7] - p[1], bz = p[8] - p[2];
    const float nx = ay * bz - az * by, ny = az * bx - ax * bz, nz = ax * by - ay * bx;
    const float nn = sqrtf(nx * nx + ny * ny + nz * nz);
    const float shade = nn > 0.f ? 0.15f + 0.85f * fabsf(-(nx * P.f[0] + ny * P.f[1] + nz * P.f[2])) / nn : 0.15f;
    int sg = 0;
    while (sg < P.nseg - 1 && t >= P.seg_end[sg]) ++sg;
    unsigned char c[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float v = fminf(fmaxf(P.rgb[sg][k] * shade, 0.f), 1.f);
        c[k] = (unsigned char)floorf(v * 255.f + 0.5f);
    }
    rgba[pix] = make_uchar4(c[0], c[1], c[2], 255);
    if (depth) depth[pix] = __uint_as_float((unsigned)(key >> 32));
}

static const float kPalette[16][3] = {
    {0.90f, 0.35f, 0.25f}, {0.25f, 0.60f, 0.90f}, {0.35f, 0.85f, 0.40f}, {0.95f, 0.80f, 0.25f},
    {0.70f, 0.40f, 0.85f}, {0.30f, 0.85f, 0.85f}, {0.95f, 0.55f, 0.75f}, {0.60f, 0.60f, 0.60f},
    {0.80f, 0.50f, 0.20f}, {0.20f, 0.40f, 0.70f}, {0.50f, 0.70f, 0.20f}, {0.90f, 0.90f, 0.90f},
    {0.55f, 0.25f, 0.45f}, {0.20f, 0.65f, 0.55f}, {0.85f, 0.30f, 0.55f}, {0.40f, 0.40f, 0.80f}};

static void unit3(double *a)
{
    const double n = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    a[0] /= n;
    a[1] /= n;
    a[2] /= n;
}

sem_status render_run(sem_ctx *ctx, const float *tris, int64_t ntri64, const int64_t *seg_ntri, int nseg,
                      const float *seg_rgb, const sem_camera *cam, int W, int H, uint8_t *rgba, float *depth)
{
    RenderParams P;
    memset(&P, 0, sizeof P);
    double f[3], s[3], u[3], up[3];
    for (int k = 0; k < 3; ++k) {
        f[k] = (double)cam->center[k] - (double)cam->eye[k];
        up[k] = cam->up[k];
    }
    unit3(f);
    s[0] = f[1] * up[2] - f[2] * up[1];
    s[1] = f[2] * up[0] - f[0] * up[2];
    s[2] = f[0] * up[1] - f[1] * up[0];
    if (!(s[0] * s[0] + s[1] * s[1] + s[2] * s[2] > 0.0))
        return sem_fail(ctx, SEM_ERR_ARG, "sem_render: up is parallel to the view direction");
    unit3(s);
    u[0] = s[1] * f[2] - s[2] * f[1];
    u[1] = s[2] * f[0] - s[0] * f[2];
    u[2] = s[0] * f[1] - s[1] * f[0];
    for (int k = 0; k < 3; ++k) {
        P.eye[k] = cam->eye[k];
        P.f[k] = (float)f[k];
        P.s[k] = (float)s[k];
        P.u[k] = (float)u[k];
    }
    const double aspect = (double)W / (double)H;
    P.ortho = cam->ortho != 0;
    if (P.ortho) {
        P.ax = (float)(1.0 / ((double)cam->half_h * aspect));
        P.ay = (float)(1.0 / (double)cam->half_h);
        P.za = (float)(1.0 / ((double)cam->zfar - (double)cam->znear));
    } else {
        const double th = tan(0.5 * (double)cam->fovy_deg * M_PI / 180.0);
        P.ax = (float)(1.0 / (th * aspect));
        P.ay = (float)(1.0 / th);
        P.zb = (float)((double)cam->zfar / ((double)cam->zfar - (double)cam->znear));
    }
    P.znear = cam->znear;
    P.zfar = cam->zfar;
    P.W = W;
    P.H = H;
    P.TW = (W + TILE - 1) / TILE;
    P.TH = (H + TILE - 1) / TILE;
    P.nseg = nseg;
    int64_t acc = 0;
    for (int k = 0; k < nseg; ++k) {
        acc += seg_ntri[k];
        P.seg_end[k] = (int)acc;
        for (int c = 0; c < 3; ++c) P.rgb[k][c] = seg_rgb ? seg_rgb[3 * k + c] : kPalette[k][c];
    }
    const int ntri = (int)ntri64;
    const int ntiles = P.TW * P.TH;

    // scratch layout: [tile_cnt | tile_cur] int32 x ntiles each, tile_off int64 x (ntiles+1),
    // scan tmp, setup records; the tile list lives in its own arena (sized after the scan)
    auto al = [](size_t b) { return ((b + 255) / 256) * 256; };
    const size_t b_cnt = al(sizeof(int32_t) * ntiles), b_off = al(sizeof(int64_t) * (ntiles + 1));
    const size_t b_tmp = al(scan_tmp_bytes(ntiles)), b_rec = al(sizeof(TriSetup) * (size_t)(ntri > 0 ? ntri : 1));
    void *scr;
    SEM_TRY(sem_scratch(ctx, SCR_RENDER, 2 * b_cnt + b_off + b_tmp + b_rec, &scr));
    char *b = reinterpret_cast<char *>(scr);
    int32_t *tile_cnt = reinterpret_cast<int32_t *>(b);
    int32_t *tile_cur = reinterpret_cast<int32_t *>(b + b_cnt);
    int64_t *tile_off = reinterpret_cast<int64_t *>(b + 2 * b_cnt);
    void *tmp = b + 2 * b_cnt + b_off;
    TriSetup *rec = reinterpret_cast<TriSetup *>(b + 2 * b_cnt + b_off + b_tmp);

    SEM_CU(ctx, cudaMemsetAsync(tile_cnt, 0, 2 * b_cnt, ctx->stream));
    if (ntri > 0) {
        k_setup<<<(ntri + 255) / 256, 256, 0, ctx->stream>>>(tris, ntri, P, rec, tile_cnt);
        SEM_CU(ctx, cudaGetLastError());
    }
    SEM_TRY(scan_i32_i64(ctx, tile_cnt, tile_off, ntiles, tmp));
    SEM_CU(ctx, cudaMemcpyAsync(ctx->h_pinned + 1, tile_off + ntiles, sizeof(int64_t), cudaMemcpyDeviceToHost,
                                ctx->stream));
    SEM_CU(ctx, cudaStreamSynchronize(ctx->stream));
    const int64_t npairs = ctx->h_pinned[1];
    void *lst;
    SEM_TRY(sem_scratch(ctx, SCR_TRI, sizeof(int32_t) * (size_t)(npairs > 0 ? npairs : 1), &lst));
    int32_t *list = reinterpret_cast<int32_t *>(lst);
    if (ntri > 0 && npairs > 0) {
        k_bin<<<(ntri + 255) / 256, 256, 0, ctx->stream>>>(rec, ntri, P.TW, tile_off, tile_cur, list);
        SEM_CU(ctx, cudaGetLastError());
    }
    k_raster<<<ntiles, RT_THREADS, 0, ctx->stream>>>(tris, rec, tile_off, list, P, reinterpret_cast<uchar4 *>(rgba), depth);
    return sem_cuda(ctx, cudaGetLastError(), "k_raster launch");
}
