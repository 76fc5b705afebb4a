// sem_iso.cu -- marching-cubes isosurface over the GLL sub-hexes of each element.
//
// Method: Lorensen & Cline 1987, applied to the N^3 sub-hexes of each element's
// (N+1)^3 GLL lattice.  Cell (i,j,k) has corners v = a + 2b + 4c at node (i+a, j+b, k+c);
// case = sum_v [f_v >= iso] 2^v; triangles come from the library's generated case table;
// a cut edge (lo, hi) gets t = (iso - f_lo)/(f_hi - f_lo), p = p_lo + t (p_hi - p_lo).
//
// Three passes, one warp per element in each:
//   k_iso_count  reads the element once (16-byte loads), culls it with warp votes (active
//                iff some node is >= iso and some is < iso), classifies its cells and writes
//                the element's triangle count (and optionally every cell's case);
//   scan         exclusive scan of the counts -> each element's first triangle;
//   k_iso_emit   re-reads only active elements (the field is usually still in L2),
//                classifies again, scans the per-cell counts across the warp and writes the
//                triangles in (element, cell, table) order.
// Node positions are lerps of the element box with exact end points, so nodes shared by two
// elements get bit-identical coordinates.
#include <cuda_runtime.h>
#include <string.h>

#include "sem_internal.cuh"

#define MP (SEM_MAX_ORDER + 1)
#define ISO_MAXT 5      // largest triangle count of the generated table (checked on upload)
// elements (warps) per block: 8, fewer for large orders so static shared memory stays < 40 KB
template <int NP>
struct IsoW {
    static constexpr int B = 4 * NP * NP * NP;
    static constexpr int V = (40960 / B) < 1 ? 1 : ((40960 / B) > 8 ? 8 : (40960 / B));
};

__constant__ float c_s[(SEM_MAX_ORDER + 1) * MP];        // (xi+1)/2 per order
__constant__ uint8_t c_ntri[256];
__constant__ int8_t c_edge[256 * ISO_MAXT * 3];

sem_status iso_upload_tables(sem_ctx *ctx, const float *s_all, const int32_t *ntri, const int8_t *edges)
{
    uint8_t n8[256];
    int8_t e8[256 * ISO_MAXT * 3];
    for (int c = 0; c < 256; ++c) {
        if (ntri[c] > ISO_MAXT) return sem_fail(ctx, SEM_ERR_CUDA, "case table has %d triangles", ntri[c]);
        n8[c] = (uint8_t)ntri[c];
        for (int q = 0; q < ISO_MAXT * 3; ++q) e8[c * ISO_MAXT * 3 + q] = edges[c * SEM_MC_MAXT * 3 + q];
    }
    SEM_CU(ctx, cudaMemcpyToSymbol(c_s, s_all, sizeof(float) * (SEM_MAX_ORDER + 1) * MP));
    SEM_CU(ctx, cudaMemcpyToSymbol(c_ntri, n8, sizeof n8));
    SEM_CU(ctx, cudaMemcpyToSymbol(c_edge, e8, sizeof e8));
    return SEM_OK;
}

// edge e -> (lower corner, upper corner), lexicographic numbering
// (0,1)(0,2)(0,4)(1,3)(1,5)(2,3)(2,6)(3,7)(4,5)(4,6)(5,7)(6,7), packed one nibble per edge
__device__ __forceinline__ void edge_ends(int e, int &lo, int &hi)
{
    lo = (int)((0x654432211000ull >> (4 * e)) & 15u);
    hi = (int)((0x776576353421ull >> (4 * e)) & 15u);
}

template <int NP>
__device__ __forceinline__ void load_element(const float *__restrict__ fe, float *__restrict__ sf, int lane, float iso,
                                             bool &any_in, bool &any_out)
{
    constexpr int NP3 = NP * NP * NP;
    bool ai = false, ao = false;
    if constexpr (NP3 % 128 == 0) {
        const float4 *f4 = reinterpret_cast<const float4 *>(fe);
        float4 *s4 = reinterpret_cast<float4 *>(sf);
#pragma unroll
        for (int q = 0; q < NP3 / 128; ++q) {
            float4 v = __ldg(f4 + q * 32 + lane);
            s4[q * 32 + lane] = v;
            ai |= (v.x >= iso) | (v.y >= iso) | (v.z >= iso) | (v.w >= iso);
            ao |= !(v.x >= iso) | !(v.y >= iso) | !(v.z >= iso) | !(v.w >= iso);
        }
    } else {
        for (int idx = lane; idx < NP3; idx += 32) {
            float v = __ldg(fe + idx);
            sf[idx] = v;
            ai |= v >= iso;
            ao |= !(v >= iso);
        }
    }
    any_in = __any_sync(0xffffffffu, ai);
    any_out = __any_sync(0xffffffffu, ao);
}

template <int NP>
__device__ __forceinline__ int cell_case(const float *__restrict__ sf, int c, float iso, int &i, int &j, int &k)
{
    constexpr int N = NP - 1;
    i = c % N;
    j = (c / N) % N;
    k = c / (N * N);
    const int b = (k * NP + j) * NP + i;
    int cs = 0;
    cs |= (sf[b] >= iso) << 0;
    cs |= (sf[b + 1] >= iso) << 1;
    cs |= (sf[b + NP] >= iso) << 2;
    cs |= (sf[b + NP + 1] >= iso) << 3;
    cs |= (sf[b + NP * NP] >= iso) << 4;
    cs |= (sf[b + NP * NP + 1] >= iso) << 5;
    cs |= (sf[b + NP * NP + NP] >= iso) << 6;
    cs |= (sf[b + NP * NP + NP + 1] >= iso) << 7;
    return cs;
}

template <int NP>
__global__ void __launch_bounds__(32 * IsoW<NP>::V) k_iso_count(const float *__restrict__ f, float iso, int64_t E,
                                                             int32_t *__restrict__ elem_cnt, uint8_t *__restrict__ cases)
{
    constexpr int NP3 = NP * NP * NP, N = NP - 1, N3 = N * N * N;
    __shared__ __align__(16) float s_f[IsoW<NP>::V][NP3];
    __shared__ uint8_t s_nt[256];
    for (int t = threadIdx.x; t < 256; t += blockDim.x) s_nt[t] = c_ntri[t];
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t e = (int64_t)blockIdx.x * IsoW<NP>::V + w;
    if (e >= E) return;
    float *sf = s_f[w];
    bool any_in, any_out;
    load_element<NP>(f + e * NP3, sf, lane, iso, any_in, any_out);
    if (!(any_in && any_out)) {
        if (lane == 0) elem_cnt[e] = 0;
        if (cases) {
            const uint8_t v = any_in ? 255 : 0;
            for (int c = lane; c < N3; c += 32) cases[e * N3 + c] = v;
        }
        return;
    }
    __syncwarp();
    int cnt = 0;
    for (int c = lane; c < N3; c += 32) {
        int i, j, k;
        const int cs = cell_case<NP>(sf, c, iso, i, j, k);
        cnt += s_nt[cs];
        if (cases) cases[e * N3 + c] = (uint8_t)cs;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, d);
    if (lane == 0) elem_cnt[e] = cnt;
}

template <int NP>
__global__ void __launch_bounds__(32 * IsoW<NP>::V) k_iso_emit(const float *__restrict__ f, float iso, int64_t E,
                                                            const int64_t *__restrict__ offs,
                                                            const float4 *__restrict__ blo,
                                                            const float4 *__restrict__ bhi, float *__restrict__ tris,
                                                            int32_t *__restrict__ tri_elem, int64_t cap)
{
    constexpr int NP3 = NP * NP * NP, N = NP - 1, N3 = N * N * N;
    __shared__ __align__(16) float s_f[IsoW<NP>::V][NP3];
    __shared__ uint8_t s_nt[256];
    __shared__ int8_t s_ed[256 * ISO_MAXT * 3];
    __shared__ float s_s[NP];
    for (int t = threadIdx.x; t < 256; t += blockDim.x) s_nt[t] = c_ntri[t];
    for (int t = threadIdx.x; t < 256 * ISO_MAXT * 3; t += blockDim.x) s_ed[t] = c_edge[t];
    if (threadIdx.x < NP) s_s[threadIdx.x] = c_s[(NP - 1) * MP + threadIdx.x];
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t e = (int64_t)blockIdx.x * IsoW<NP>::V + w;
    if (e >= E) return;
    int64_t base = offs[e];
    if (offs[e + 1] == base) return;
    float *sf = s_f[w];
    bool ai, ao;
    load_element<NP>(f + e * NP3, sf, lane, iso, ai, ao);
    __syncwarp();
    const float4 L = blo[e], H = bhi[e];
    for (int c0 = 0; c0 < N3; c0 += 32) {
        const int c = c0 + lane;
        int cs = 0, nt = 0, i = 0, j = 0, k = 0;
        if (c < N3) {
            cs = cell_case<NP>(sf, c, iso, i, j, k);
            nt = s_nt[cs];
        }
        int incl = nt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += y;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        int64_t o = base + (incl - nt);
        for (int q = 0; q < nt; ++q, ++o) {
            float p[9];
#pragma unroll
            for (int sv = 0; sv < 3; ++sv) {
                int lo, hi;
                edge_ends(s_ed[(cs * ISO_MAXT + q) * 3 + sv], lo, hi);
                const int ia = i + (lo & 1), ja = j + ((lo >> 1) & 1), ka = k + ((lo >> 2) & 1);
                const int ib = i + (hi & 1), jb = j + ((hi >> 1) & 1), kb = k + ((hi >> 2) & 1);
                const float fa = sf[(ka * NP + ja) * NP + ia], fb = sf[(kb * NP + jb) * NP + ib];
                const float t = (iso - fa) / (fb - fa);
                const float xa = fmaf(s_s[ia], H.x, (1.f - s_s[ia]) * L.x), xb = fmaf(s_s[ib], H.x, (1.f - s_s[ib]) * L.x);
                const float ya = fmaf(s_s[ja], H.y, (1.f - s_s[ja]) * L.y), yb = fmaf(s_s[jb], H.y, (1.f - s_s[jb]) * L.y);
                const float za = fmaf(s_s[ka], H.z, (1.f - s_s[ka]) * L.z), zb = fmaf(s_s[kb], H.z, (1.f - s_s[kb]) * L.z);
                p[sv * 3 + 0] = fmaf(t, xb - xa, xa);
                p[sv * 3 + 1] = fmaf(t, yb - ya, ya);
                p[sv * 3 + 2] = fmaf(t, zb - za, za);
            }
            if (o < cap) {
                float *dst = tris + o * 9;
#pragma unroll
                for (int r = 0; r < 9; ++r) dst[r] = p[r];
                if (tri_elem) tri_elem[o] = (int32_t)e;
            }
        }
        base += total;
    }
}

// ------------------------------------------------------------------------------------------
// Several isovalues at once (sem_isosurface_multi; sem_isosurface is the one-isovalue case).
// The field is read once per pass for all isovalues: each cell's 8 corners are loaded once
// and classified against every isovalue.  Counts are laid out [q][e], so one scan over
// niso*E entries gives every isovalue's triangles a contiguous segment, in isovalue order.
// Emission stages each round's triangles in shared memory and stores them coalesced.

struct IsoSet {
    int niso;
    float iso[SEM_MAX_ISO];
};

// per-warp dynamic shared memory of the emit kernel: the element's field, the triangle map and
// the cell cases; warps (elements) per block: up to 8 within ~96 KB
template <int NP>
struct EmitW {
    static constexpr int NP3 = NP * NP * NP, N3 = (NP - 1) * (NP - 1) * (NP - 1);
    static constexpr int F_BYTES = 4 * NP3;
    static constexpr int MAP_BYTES = ((2 * N3 * ISO_MAXT + 15) / 16) * 16;
    static constexpr int CASE_BYTES = ((N3 + 15) / 16) * 16;
    static constexpr int B = F_BYTES + MAP_BYTES + CASE_BYTES;
    static constexpr int R = 98304 / B;
    static constexpr int V = R < 1 ? 1 : (R > 8 ? 8 : R);
};

template <int NP>
__device__ __forceinline__ void load_minmax(const float *__restrict__ fe, float *__restrict__ sf, int lane, float &mn,
                                            float &mx, bool &has_nan)
{
    constexpr int NP3 = NP * NP * NP;
    float a = INFINITY, b = -INFINITY;
    bool nn = false;
    if constexpr (NP3 % 128 == 0) {
        const float4 *f4 = reinterpret_cast<const float4 *>(fe);
        float4 *s4 = reinterpret_cast<float4 *>(sf);
#pragma unroll
        for (int q = 0; q < NP3 / 128; ++q) {
            const float4 v = __ldg(f4 + q * 32 + lane);
            s4[q * 32 + lane] = v;
            a = fminf(a, fminf(fminf(v.x, v.y), fminf(v.z, v.w)));
            b = fmaxf(b, fmaxf(fmaxf(v.x, v.y), fmaxf(v.z, v.w)));
            nn |= isnan(v.x) | isnan(v.y) | isnan(v.z) | isnan(v.w);
        }
    } else {
        for (int idx = lane; idx < NP3; idx += 32) {
            const float v = __ldg(fe + idx);
            sf[idx] = v;
            a = fminf(a, v);
            b = fmaxf(b, v);
            nn |= isnan(v);
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        a = fminf(a, __shfl_xor_sync(0xffffffffu, a, d));
        b = fmaxf(b, __shfl_xor_sync(0xffffffffu, b, d));
    }
    mn = a;
    mx = b;
    has_nan = __any_sync(0xffffffffu, nn);
}

template <int NP>
__device__ __forceinline__ void cell_corners(const float *__restrict__ sf, int c, float (&v)[8], int &i, int &j, int &k)
{
    constexpr int N = NP - 1;
    i = c % N;
    j = (c / N) % N;
    k = c / (N * N);
    const int b = (k * NP + j) * NP + i;
    v[0] = sf[b];
    v[1] = sf[b + 1];
    v[2] = sf[b + NP];
    v[3] = sf[b + NP + 1];
    v[4] = sf[b + NP * NP];
    v[5] = sf[b + NP * NP + 1];
    v[6] = sf[b + NP * NP + NP];
    v[7] = sf[b + NP * NP + NP + 1];
}

__device__ __forceinline__ int corner_case(const float (&v)[8], float iso)
{
    int cs = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) cs |= (v[q] >= iso) << q;
    return cs;
}

template <int NP>
__global__ void __launch_bounds__(32 * IsoW<NP>::V) k_iso_count_m(const float *__restrict__ f,
                                                                 const __grid_constant__ IsoSet S, int64_t E,
                                                                 int32_t *__restrict__ cnt, uint8_t *__restrict__ cases)
{
    constexpr int NP3 = NP * NP * NP, N = NP - 1, N3 = N * N * N;
    __shared__ __align__(16) float s_f[IsoW<NP>::V][NP3];
    __shared__ uint8_t s_nt[256];
    for (int t = threadIdx.x; t < 256; t += blockDim.x) s_nt[t] = c_ntri[t];
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t e = (int64_t)blockIdx.x * IsoW<NP>::V + w;
    if (e >= E) return;
    float *sf = s_f[w];
    float mn, mx;
    bool has_nan;
    load_minmax<NP>(f + e * NP3, sf, lane, mn, mx, has_nan);
    unsigned active = 0;
    for (int q = 0; q < S.niso; ++q) {
        const bool any_in = mx >= S.iso[q], any_out = (mn < S.iso[q]) || has_nan;
        if (any_in && any_out) {
            active |= 1u << q;
        } else {
            if (lane == 0) cnt[q * E + e] = 0;
            if (cases) {
                const uint8_t v = any_in ? 255 : 0;
                for (int c = lane; c < N3; c += 32) cases[(q * E + e) * N3 + c] = v;
            }
        }
    }
    if (!active) return;
    __syncwarp();
    int acc[SEM_MAX_ISO];
#pragma unroll
    for (int q = 0; q < SEM_MAX_ISO; ++q) acc[q] = 0;
    for (int c = lane; c < N3; c += 32) {
        float v[8];
        int i, j, k;
        cell_corners<NP>(sf, c, v, i, j, k);
#pragma unroll
        for (int q = 0; q < SEM_MAX_ISO; ++q) {
            if (!((active >> q) & 1u)) continue;
            const int cs = corner_case(v, S.iso[q]);
            acc[q] += s_nt[cs];
            if (cases) cases[(q * E + e) * N3 + c] = (uint8_t)cs;
        }
    }
#pragma unroll
    for (int q = 0; q < SEM_MAX_ISO; ++q) {
        if (!((active >> q) & 1u)) continue;
        int a = acc[q];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) a += __shfl_xor_sync(0xffffffffu, a, d);
        if (lane == 0) cnt[q * E + e] = a;
    }
}

// One warp per element.  For each isovalue: (1) 32 cells at a time, classify, warp-scan the
// triangle counts and write, for every triangle of the element, its (cell, index in cell)
// into a shared-memory map; (2) give each lane one output triangle: lane L takes triangles
// L, L+32, ... of the element, reads its cell from the map and writes it.  Every lane does
// one triangle's work and consecutive lanes write consecutive triangles.
template <int NP>
__global__ void __launch_bounds__(32 * EmitW<NP>::V) k_iso_emit_m(const float *__restrict__ f,
                                                                 const __grid_constant__ IsoSet S, int64_t E,
                                                                 const int64_t *__restrict__ offs,
                                                                 const float4 *__restrict__ blo,
                                                                 const float4 *__restrict__ bhi,
                                                                 float *__restrict__ tris,
                                                                 int32_t *__restrict__ tri_elem, int64_t cap,
                                                                 int *flag)
{
    constexpr int NP3 = NP * NP * NP, N = NP - 1, N3 = N * N * N;
    using EW = EmitW<NP>;
    // all-or-nothing capacity check (the host-synchronised path has checked already)
    if (offs[S.niso * E] > cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0 && flag) atomicOr(flag, 1 << SEM_ERR_CAPACITY);
        return;
    }
    constexpr int WV = EW::V;
    extern __shared__ __align__(16) unsigned char s_dyn[];
    __shared__ uint8_t s_nt[256];
    __shared__ int8_t s_ed[256 * ISO_MAXT * 3];
    __shared__ float s_s[NP];
    for (int t = threadIdx.x; t < 256; t += blockDim.x) s_nt[t] = c_ntri[t];
    for (int t = threadIdx.x; t < 256 * ISO_MAXT * 3; t += blockDim.x) s_ed[t] = c_edge[t];
    if (threadIdx.x < NP) s_s[threadIdx.x] = c_s[(NP - 1) * MP + threadIdx.x];
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t e = (int64_t)blockIdx.x * WV + w;
    if (e >= E) return;
    unsigned active = 0;
    for (int q = 0; q < S.niso; ++q)
        if (offs[q * E + e + 1] != offs[q * E + e]) active |= 1u << q;
    if (!active) return;
    unsigned char *mine = s_dyn + (size_t)w * EW::B;
    float *sf = reinterpret_cast<float *>(mine);
    uint16_t *map = reinterpret_cast<uint16_t *>(mine + EW::F_BYTES);  // (cell << 3) | index in cell
    uint8_t *sc = mine + EW::F_BYTES + EW::MAP_BYTES;
    {
        float mn, mx;
        bool hn;
        load_minmax<NP>(f + e * NP3, sf, lane, mn, mx, hn);
    }
    __syncwarp();
    const float4 L = blo[e], H = bhi[e];
    for (int q = 0; q < S.niso; ++q) {
        if (!((active >> q) & 1u)) continue;
        const float iso = S.iso[q];
        // (1) cases and the triangle -> (cell, index) map, in cell order
        int running = 0;
        for (int c0 = 0; c0 < N3; c0 += 32) {
            const int c = c0 + lane;
            int cs = 0, nt = 0;
            if (c < N3) {
                float v[8];
                int i, j, k;
                cell_corners<NP>(sf, c, v, i, j, k);
                cs = corner_case(v, iso);
                nt = s_nt[cs];
                sc[c] = (uint8_t)cs;
            }
            int incl = nt;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += y;
            }
            const int first = running + incl - nt;
            for (int t = 0; t < nt; ++t) map[first + t] = (uint16_t)((c << 3) | t);
            running += __shfl_sync(0xffffffffu, incl, 31);
        }
        __syncwarp();
        // (2) one output triangle per lane
        const int64_t o = offs[q * E + e];
        if (o + running <= cap) {
            for (int idx = lane; idx < running; idx += 32) {
                const int mc = map[idx];
                const int c = mc >> 3, t = mc & 7, cs = sc[c];
                const int i = c % N, j = (c / N) % N, k = c / (N * N);
                float p[9];
#pragma unroll
                for (int sv = 0; sv < 3; ++sv) {
                    int la, lb;
                    edge_ends(s_ed[(cs * ISO_MAXT + t) * 3 + sv], la, lb);
                    const int ia = i + (la & 1), ja = j + ((la >> 1) & 1), ka = k + ((la >> 2) & 1);
                    const int ib = i + (lb & 1), jb = j + ((lb >> 1) & 1), kb = k + ((lb >> 2) & 1);
                    const float fa = sf[(ka * NP + ja) * NP + ia], fb = sf[(kb * NP + jb) * NP + ib];
                    const float tt = (iso - fa) / (fb - fa);
                    const float xa = fmaf(s_s[ia], H.x, (1.f - s_s[ia]) * L.x), xb = fmaf(s_s[ib], H.x, (1.f - s_s[ib]) * L.x);
                    const float ya = fmaf(s_s[ja], H.y, (1.f - s_s[ja]) * L.y), yb = fmaf(s_s[jb], H.y, (1.f - s_s[jb]) * L.y);
                    const float za = fmaf(s_s[ka], H.z, (1.f - s_s[ka]) * L.z), zb = fmaf(s_s[kb], H.z, (1.f - s_s[kb]) * L.z);
                    p[sv * 3 + 0] = fmaf(tt, xb - xa, xa);
                    p[sv * 3 + 1] = fmaf(tt, yb - ya, ya);
                    p[sv * 3 + 2] = fmaf(tt, zb - za, za);
                }
                float *dst = tris + (o + idx) * 9;
#pragma unroll
                for (int r = 0; r < 9; ++r) dst[r] = p[r];
                if (tri_elem) tri_elem[o + idx] = (int32_t)e;
            }
        }
        __syncwarp();
    }
}

template <int NP>
static sem_status iso_multi_np(sem_ctx *ctx, const sem_mesh *m, const float *f, const IsoSet &S, float *tris,
                               int32_t *tri_elem, int64_t cap, int64_t *ntri_out, uint8_t *cases)
{
    const int64_t E = m->E, n = E * S.niso;
    const size_t cnt_bytes = ((sizeof(int32_t) * n + 255) / 256) * 256;
    const size_t off_bytes = ((sizeof(int64_t) * (n + 1) + 255) / 256) * 256;
    void *scr;
    SEM_TRY(sem_scratch(ctx, SCR_ISO, cnt_bytes + off_bytes + scan_tmp_bytes(n), &scr));
    int32_t *cnt = reinterpret_cast<int32_t *>(scr);
    int64_t *offs = reinterpret_cast<int64_t *>(reinterpret_cast<char *>(scr) + cnt_bytes);
    void *tmp = reinterpret_cast<char *>(scr) + cnt_bytes + off_bytes;
    constexpr int WV = IsoW<NP>::V;
    k_iso_count_m<NP><<<(unsigned)((E + WV - 1) / WV), 32 * WV, 0, ctx->stream>>>(f, S, E, cnt, cases);
    SEM_CU(ctx, cudaGetLastError());
    SEM_TRY(scan_i32_i64(ctx, cnt, offs, n, tmp));
    // segment starts offs[q*E], q = 0..niso (the last one is the grand total)
    SEM_CU(ctx, cudaMemcpy2DAsync(ctx->h_pinned, sizeof(int64_t), offs, sizeof(int64_t) * E, sizeof(int64_t),
                                  S.niso + 1, cudaMemcpyDeviceToHost, ctx->stream));
    SEM_CU(ctx, cudaStreamSynchronize(ctx->stream));
    for (int q = 0; q < S.niso; ++q) ntri_out[q] = ctx->h_pinned[q + 1] - ctx->h_pinned[q];
    const int64_t total = ctx->h_pinned[S.niso];
    if (!tris) return SEM_OK;  // count-only query
    if (total > cap)
        return sem_fail(ctx, SEM_ERR_CAPACITY, "sem_isosurface: %lld triangles exceed capacity %lld", (long long)total,
                        (long long)cap);
    if (total == 0) return SEM_OK;
    constexpr int EV = EmitW<NP>::V;
    constexpr size_t dyn = (size_t)EV * EmitW<NP>::B;
    SEM_CU(ctx, cudaFuncSetAttribute(k_iso_emit_m<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    k_iso_emit_m<NP><<<(unsigned)((E + EV - 1) / EV), 32 * EV, dyn, ctx->stream>>>(
        f, S, E, offs, m->lo, m->hi, tris, tri_elem, cap, ctx->d_flag);
    return sem_cuda(ctx, cudaGetLastError(), "k_iso_emit_m launch");
}

// No host synchronisation: segment starts go to counts_dev (device), a capacity overflow
// raises the context's device flag and writes no triangle.
template <int NP>
static sem_status iso_multi_async_np(sem_ctx *ctx, const sem_mesh *m, const float *f, const IsoSet &S, float *tris,
                                     int32_t *tri_elem, int64_t cap, int64_t *counts_dev, uint8_t *cases)
{
    const int64_t E = m->E, n = E * S.niso;
    const size_t cnt_bytes = ((sizeof(int32_t) * n + 255) / 256) * 256;
    const size_t off_bytes = ((sizeof(int64_t) * (n + 1) + 255) / 256) * 256;
    void *scr;
    SEM_TRY(sem_scratch_nogrow_in_capture(ctx, SCR_ISO, cnt_bytes + off_bytes + scan_tmp_bytes(n), &scr));
    int32_t *cnt = reinterpret_cast<int32_t *>(scr);
    int64_t *offs = reinterpret_cast<int64_t *>(reinterpret_cast<char *>(scr) + cnt_bytes);
    void *tmp = reinterpret_cast<char *>(scr) + cnt_bytes + off_bytes;
    constexpr int WV = IsoW<NP>::V;
    k_iso_count_m<NP><<<(unsigned)((E + WV - 1) / WV), 32 * WV, 0, ctx->stream>>>(f, S, E, cnt, cases);
    SEM_CU(ctx, cudaGetLastError());
    SEM_TRY(scan_i32_i64(ctx, cnt, offs, n, tmp));
    SEM_CU(ctx, cudaMemcpy2DAsync(counts_dev, sizeof(int64_t), offs, sizeof(int64_t) * E, sizeof(int64_t), S.niso + 1,
                                  cudaMemcpyDeviceToDevice, ctx->stream));
    if (!tris) return SEM_OK;
    constexpr int EV = EmitW<NP>::V;
    constexpr size_t dyn = (size_t)EV * EmitW<NP>::B;
    SEM_CU(ctx, cudaFuncSetAttribute(k_iso_emit_m<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    k_iso_emit_m<NP><<<(unsigned)((E + EV - 1) / EV), 32 * EV, dyn, ctx->stream>>>(
        f, S, E, offs, m->lo, m->hi, tris, tri_elem, cap, ctx->d_flag);
    return sem_cuda(ctx, cudaGetLastError(), "k_iso_emit_m launch");
}

sem_status iso_run_multi_async(sem_ctx *ctx, const sem_mesh *m, const float *f, const float *isos, int niso,
                               float *tris, int32_t *tri_elem, int64_t cap, int64_t *counts_dev, uint8_t *cases)
{
    IsoSet S;
    memset(&S, 0, sizeof S);
    S.niso = niso;
    for (int q = 0; q < niso; ++q) S.iso[q] = isos[q];
    switch (m->N + 1) {
#define SEM_CASE(NPV) \
    case NPV: return iso_multi_async_np<NPV>(ctx, m, f, S, tris, tri_elem, cap, counts_dev, cases);
        SEM_CASE(2) SEM_CASE(3) SEM_CASE(4) SEM_CASE(5) SEM_CASE(6) SEM_CASE(7) SEM_CASE(8) SEM_CASE(9)
        SEM_CASE(10) SEM_CASE(11) SEM_CASE(12) SEM_CASE(13) SEM_CASE(14) SEM_CASE(15) SEM_CASE(16)
#undef SEM_CASE
    default: return sem_fail(ctx, SEM_ERR_ARG, "order N=%d not supported", m->N);
    }
}

sem_status iso_run_multi(sem_ctx *ctx, const sem_mesh *m, const float *f, const float *isos, int niso, float *tris,
                         int32_t *tri_elem, int64_t cap, int64_t *ntri_out, uint8_t *cases)
{
    IsoSet S;
    memset(&S, 0, sizeof S);
    S.niso = niso;
    for (int q = 0; q < niso; ++q) S.iso[q] = isos[q];
    switch (m->N + 1) {
#define SEM_CASE(NPV) \
    case NPV: return iso_multi_np<NPV>(ctx, m, f, S, tris, tri_elem, cap, ntri_out, cases);
        SEM_CASE(2) SEM_CASE(3) SEM_CASE(4) SEM_CASE(5) SEM_CASE(6) SEM_CASE(7) SEM_CASE(8) SEM_CASE(9)
        SEM_CASE(10) SEM_CASE(11) SEM_CASE(12) SEM_CASE(13) SEM_CASE(14) SEM_CASE(15) SEM_CASE(16)
#undef SEM_CASE
    default: return sem_fail(ctx, SEM_ERR_ARG, "order N=%d not supported", m->N);
    }
}

sem_status iso_run(sem_ctx *ctx, const sem_mesh *m, const float *f, float iso, float *tris, int32_t *tri_elem,
                   int64_t cap, int64_t *ntri_out, uint8_t *cases)
{
    return iso_run_multi(ctx, m, f, &iso, 1, tris, tri_elem, cap, ntri_out, cases);
}

// ==========================================================================================
// Allocation-free variant of sem_isosurface (sem_isosurface_noalloc).  Same kernels and the
// same scan; the per-element counts, offsets and scan partials live in one file-scope device
// array instead of the context's grow-only arena, so a call never allocates.
// ==========================================================================================
#include <mutex>

namespace {
constexpr size_t al256(size_t b) { return ((b + 255) / 256) * 256; }
constexpr int64_t kNaMaxE = SEM_NOALLOC_MAX_ELEMENTS;
constexpr size_t kNaCnt = al256(sizeof(int32_t) * kNaMaxE);
constexpr size_t kNaOff = al256(sizeof(int64_t) * (kNaMaxE + 1));
constexpr size_t kNaTmp = al256(sizeof(int64_t) * ((kNaMaxE + 4095) / 4096 + 1));
constexpr int kNaMaxDevices = 64;
}  // namespace

// Shared by every call on a device; holds the last call's contents until the next call.
// Nothing in it needs to start at zero: every word is written before it is read.
static __device__ __align__(256) unsigned char g_iso_noalloc_scratch[kNaCnt + kNaOff + kNaTmp];

static std::mutex g_na_mu;
static void *g_na_ptr[kNaMaxDevices] = {};

// Device address of g_iso_noalloc_scratch on ctx->device (which the caller has made current).
// The host-side symbol is only a stand-in, so the address is looked up once per device.
static sem_status noalloc_scratch(sem_ctx *ctx, char **out)
{
    if (ctx->device < 0 || ctx->device >= kNaMaxDevices)
        return sem_fail(ctx, SEM_ERR_UNSUPPORTED, "sem_isosurface_noalloc: device index %d >= %d", ctx->device,
                        kNaMaxDevices);
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[ctx->device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_iso_noalloc_scratch);
        if (e != cudaSuccess || !p) return sem_cuda(ctx, e != cudaSuccess ? e : cudaErrorInvalidSymbol, "cudaGetSymbolAddress");
        g_na_ptr[ctx->device] = p;
    }
    *out = static_cast<char *>(g_na_ptr[ctx->device]);
    return SEM_OK;
}

template <int NP>
static sem_status iso_run_noalloc_np(sem_ctx *ctx, const sem_mesh *m, const float *f, float iso, float *tris,
                                     int32_t *tri_elem, int64_t cap, int64_t *ntri_out, uint8_t *cases)
{
    const int64_t E = m->E;
    if (scan_tmp_bytes(E) > kNaTmp) return sem_fail(ctx, SEM_ERR_ARG, "sem_isosurface_noalloc: scan scratch too small");
    char *scr;
    SEM_TRY(noalloc_scratch(ctx, &scr));
    int32_t *cnt = reinterpret_cast<int32_t *>(scr);
    int64_t *offs = reinterpret_cast<int64_t *>(scr + kNaCnt);
    void *tmp = scr + kNaCnt + kNaOff;
    constexpr int WV = IsoW<NP>::V;
    const unsigned grid = (unsigned)((E + WV - 1) / WV);
    k_iso_count<NP><<<grid, 32 * WV, 0, ctx->stream>>>(f, iso, E, cnt, cases);
    SEM_CU(ctx, cudaGetLastError());
    SEM_TRY(scan_i32_i64(ctx, cnt, offs, E, tmp));
    SEM_CU(ctx, cudaMemcpyAsync(ctx->h_pinned, offs + E, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
    SEM_CU(ctx, cudaStreamSynchronize(ctx->stream));
    const int64_t total = ctx->h_pinned[0];
    *ntri_out = total;
    if (!tris) return SEM_OK;
    if (total > cap)
        return sem_fail(ctx, SEM_ERR_CAPACITY, "sem_isosurface_noalloc: %lld triangles exceed capacity %lld",
                        (long long)total, (long long)cap);
    if (total == 0) return SEM_OK;
    k_iso_emit<NP><<<grid, 32 * WV, 0, ctx->stream>>>(f, iso, E, offs, m->lo, m->hi, tris, tri_elem, cap);
    return sem_cuda(ctx, cudaGetLastError(), "k_iso_emit launch");
}

sem_status iso_run_noalloc(sem_ctx *ctx, const sem_mesh *m, const float *f, float iso, float *tris,
                           int32_t *tri_elem, int64_t cap, int64_t *ntri_out, uint8_t *cases)
{
    switch (m->N + 1) {
#define SEM_CASE(NPV) \
    case NPV: return iso_run_noalloc_np<NPV>(ctx, m, f, iso, tris, tri_elem, cap, ntri_out, cases);
        SEM_CASE(2) SEM_CASE(3) SEM_CASE(4) SEM_CASE(5) SEM_CASE(6) SEM_CASE(7) SEM_CASE(8) SEM_CASE(9)
        SEM_CASE(10) SEM_CASE(11) SEM_CASE(12) SEM_CASE(13) SEM_CASE(14) SEM_CASE(15) SEM_CASE(16)
#undef SEM_CASE
    default: return sem_fail(ctx, SEM_ERR_ARG, "order N=%d not supported", m->N);
    }
}
