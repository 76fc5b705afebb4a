// sem_qcrit.cu -- spectral derivative and Q-criterion kernels (FP32, the plain path).
//
// Per element of order N the three reference derivatives are tensor-product contractions
// with the GLL collocation derivative matrix D (Canuto et al., Spectral Methods, Sec. 2.3):
//   u_r[k][j][i] = sum_m D[i][m] u[k][j][m],  u_s = sum_m D[j][m] u[k][m][i],
//   u_t = sum_m D[k][m] u[m][j][i]
// and on an affine box du/dx = (2/hx) u_r, du/dy = (2/hy) u_s, du/dz = (2/hz) u_t.
// Q = -1/2 sum_ij J_ij J_ji with J_ij = du_i/dx_j (Hunt, Wray & Moin 1988).
//
// Design (GB300): the kernel is HBM-bound (16 B of traffic per node for Q, 144 FLOP per node:
// about 9 FLOP/B, at the FP32 FFMA ridge), so it streams elements through shared memory with
// the TMA engine (cp.async.bulk, double-buffered, mbarrier completion) in a persistent grid,
// keeps D in constant memory (FFMA operands straight from the constant bank).  Every kernel
// gives each thread one r-, one s- and one t-line of (N+1) nodes of one element, so that every
// shared-memory value is read once per direction.  The derivative kernel (k_sem_grad) writes
// each line's derivatives straight to its output field; in the Q kernels (k_sem_q8 for N = 7,
// k_sem_qd for the other orders) the s- and t-derivatives reach the r-line's owner through an
// exchange buffer, which folds the six products of Q in registers and writes them.  Tensor cores are not
// used here: the contractions have K = N+1 = 8, and the element data would have to be
// transposed between the three directions, costing more shared-memory traffic than the
// FFMA work they would replace.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "sem_internal.cuh"

#define MP (SEM_MAX_ORDER + 1)

__constant__ float c_D[(SEM_MAX_ORDER + 1) * MP * MP];  // [N][i][m], FP32

// Even/odd coefficients of D for N = 7: {(D[i][m] + D[i][7-m])/2, (D[i][m] - D[i][7-m])/2} for
// i, m < 4.  GLL D is centro-antisymmetric, D[7-i][7-m] = -D[i][m], so with e_m = u_m + u_{7-m}
// and o_m = u_m - u_{7-m}:  (Du)_i = E_i + O_i and (Du)_{7-i} = O_i - E_i, where
// E_i = sum_m Ae[i][m] e_m and O_i = sum_m Ao[i][m] o_m (m < 4): 48 operations instead of 64.
__constant__ float2 c_Deo7[4 * 4];
// D transposed, [N][m][i]: the coefficients (D[i][m], D[i+1][m]) of two nodes' sums side by side
// (8-byte aligned for even i), one FFMA2 operand
__constant__ __align__(16) float c_DT[(SEM_MAX_ORDER + 1) * MP * MP];

sem_status qcrit_upload_tables(sem_ctx *ctx, const float *D_all, const float *s_all)
{
    (void)s_all;
    SEM_CU(ctx, cudaMemcpyToSymbol(c_D, D_all, sizeof(float) * (SEM_MAX_ORDER + 1) * MP * MP));
    float2 eo[16];
    const float *D7 = D_all + 7 * MP * MP;
    for (int i = 0; i < 4; ++i)
        for (int m = 0; m < 4; ++m) {
            const double a = D7[i * MP + m], b = D7[i * MP + 7 - m];
            eo[i * 4 + m] = make_float2((float)(0.5 * (a + b)), (float)(0.5 * (a - b)));
        }
    SEM_CU(ctx, cudaMemcpyToSymbol(c_Deo7, eo, sizeof eo));
    std::vector<float> dt((size_t)(SEM_MAX_ORDER + 1) * MP * MP);
    for (int n = 0; n <= SEM_MAX_ORDER; ++n)
        for (int i = 0; i < MP; ++i)
            for (int m = 0; m < MP; ++m) dt[((size_t)n * MP + m) * MP + i] = D_all[((size_t)n * MP + i) * MP + m];
    SEM_CU(ctx, cudaMemcpyToSymbol(c_DT, dt.data(), sizeof(float) * dt.size()));
    return SEM_OK;
}

template <int NP>
__device__ __forceinline__ float Dc(int i, int m)
{
    return c_D[((NP - 1) * MP + i) * MP + m];
}

// Every contraction below subtracts the line's first value from the line before the products
// (the line's level shift): D's rows sum to zero (D 1 = 0), so the derivative is unchanged in
// exact arithmetic, while the FP32 rounding then follows the field's variation along the line
// instead of its magnitude -- a field with a large mean over thin elements would otherwise
// lose most of its significant digits to cancellation.

template <int NP>
__device__ __forceinline__ float2 DT2(int m, int i)
{
    return *reinterpret_cast<const float2 *>(&c_DT[((NP - 1) * MP + m) * MP + i]);
}

// (D u)_i for i = 0..NP-1 of one line u held in registers (u is shifted in place); two nodes'
// sums share one FFMA2 (two round-to-nearest FMAs per instruction)
template <int NP>
__device__ __forceinline__ void contract_line2(float (&u)[NP], float (&d)[NP])
{
#pragma unroll
    for (int m = 1; m < NP; ++m) u[m] -= u[0];
#pragma unroll
    for (int i = 0; i + 1 < NP; i += 2) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int m = 1; m < NP; ++m) acc = __ffma2_rn(DT2<NP>(m, i), make_float2(u[m], u[m]), acc);
        d[i] = acc.x;
        d[i + 1] = acc.y;
    }
    if constexpr (NP & 1) {
        float acc = 0.f;
#pragma unroll
        for (int m = 1; m < NP; ++m) acc = fmaf(Dc<NP>(NP - 1, m), u[m], acc);
        d[NP - 1] = acc;
    }
}

// NP consecutive floats of shared memory (16- or 8-byte loads where NP allows)
template <int NP>
__device__ __forceinline__ void load_row(const float *__restrict__ src, float (&v)[NP])
{
    if constexpr (NP % 4 == 0) {
        const float4 *p = reinterpret_cast<const float4 *>(src);
#pragma unroll
        for (int q = 0; q < NP / 4; ++q) {
            const float4 x = p[q];
            v[4 * q] = x.x; v[4 * q + 1] = x.y; v[4 * q + 2] = x.z; v[4 * q + 3] = x.w;
        }
    } else if constexpr (NP % 2 == 0) {
        const float2 *p = reinterpret_cast<const float2 *>(src);
#pragma unroll
        for (int q = 0; q < NP / 2; ++q) {
            const float2 x = p[q];
            v[2 * q] = x.x; v[2 * q + 1] = x.y;
        }
    } else {
#pragma unroll
        for (int m = 0; m < NP; ++m) v[m] = src[m];
    }
}

template <int NP>
__device__ __forceinline__ void store_line(float *__restrict__ dst, const float (&v)[NP])
{
    if constexpr (NP % 4 == 0) {
        float4 *p = reinterpret_cast<float4 *>(dst);
#pragma unroll
        for (int q = 0; q < NP / 4; ++q) p[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    } else if constexpr (NP % 2 == 0) {
        float2 *p = reinterpret_cast<float2 *>(dst);
#pragma unroll
        for (int q = 0; q < NP / 2; ++q) p[q] = make_float2(v[2 * q], v[2 * q + 1]);
    } else {
#pragma unroll
        for (int i = 0; i < NP; ++i) dst[i] = v[i];
    }
}

template <int NP>
struct QCfg {
    static constexpr int L = NP * NP;
    static constexpr int NP3 = NP * NP * NP;
    static constexpr bool BULK = (NP % 2) == 0;  // element byte size is a multiple of 16
    static constexpr int EPB_RAW = (256 / L) > 0 ? (256 / L) : 1;
    static constexpr int EPB = EPB_RAW;
    static constexpr int NT = ((EPB * L + 31) / 32) * 32;
    static constexpr int NSTAGE = BULK ? 2 : 1;
#ifndef SEM_Q_MINB
#define SEM_Q_MINB 2
#endif
    // resident blocks the register allocation is sized for: N = 5 (4 blocks of 252 threads at 64
    // registers, no spills) and N = 9 (3 blocks of 224 threads) run more warps than at the
    // compiler's own choice (2 blocks each)
    static constexpr int MINB = (NP == 8) ? SEM_Q_MINB : (NP == 6 ? 4 : (NP == 10 ? 3 : 1));
};

// The partitions one launch covers (one partition for sem_qcriterion / sem_derivatives, up to
// QB_MAX of the same order for sem_qcriterion_batch).  Elements are taken in groups of EPB per
// partition; gstart[p] is partition p's first group in the launch's group numbering.
#define QB_MAX 48
struct GBatch {
    int n;
    long long wait_limit;  // polls of a wait for the stage's input copies before giving up
    int64_t gstart[QB_MAX + 1];
    int64_t E[QB_MAX];
    const float *f[3][QB_MAX];
    float *o[3][QB_MAX];
    const float4 *g[QB_MAX];
    // k_sem_q8<true> only (one partition): isovalues of Q whose per-element triangle counts the
    // kernel also writes, cnt[q E + e], and the case table's triangle counts (256 bytes)
    int niso;
    float iso[SEM_MAX_ISO];
    int32_t *cnt;
    const uint8_t *ntri;
};

// the partition holding group grp (largest p with gstart[p] <= grp)
__device__ __forceinline__ int qb_find(const GBatch &B, int64_t grp)
{
    int lo = 0, hi = B.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (B.gstart[mid] <= grp) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The gradient of f0 -> (out0, out1, out2) with direction-owned lines: thread (el, l) of a
// stage, with (a, b) = (l / NP, l % NP), contracts the r-line (k, j) = (a, b), the s-line
// (k, i) = (a, b) and the t-line (j, i) = (a, b) of element el, reading NP values per line, and
// writes each line's derivatives, scaled by the element's factor, straight to its own output
// field: rows for d/dr, runs of NP nodes for d/ds, and for d/dt stores that are contiguous
// across the threads of a warp.  No exchange and one barrier per stage after the stage's own.
template <int NP>
__global__ void __launch_bounds__(QCfg<NP>::NT, QCfg<NP>::MINB) k_sem_grad(const __grid_constant__ GBatch B, int *err)
{
    using C = QCfg<NP>;
    constexpr int NP3 = C::NP3, L = C::L, EPB = C::EPB;
    constexpr int STAGE = EPB * NP3;
    constexpr uint32_t BYTES = EPB * NP3 * 4;
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int s_abort;

    const int tid = threadIdx.x;
    const bool active = tid < EPB * L;
    const int el = active ? tid / L : 0, l = tid % L, a = l / NP, b = l % NP;
    const int64_t ngroups = B.gstart[B.n];
    // group -> (partition, its elements): a full group (EPB elements) can come by bulk copy
    auto elems = [&](int64_t grp, int &p, int64_t &e0) {
        p = qb_find(B, grp);
        e0 = (grp - B.gstart[p]) * EPB;
        const int64_t left = B.E[p] - e0;
        return (int)(left < EPB ? left : EPB);
    };
    if (tid == 0) {
        s_abort = 0;
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();

    auto full = [&](int64_t grp) {
        int p;
        int64_t e0;
        return C::BULK && grp < ngroups && elems(grp, p, e0) == EPB;
    };
    auto issue = [&](int64_t grp, int s) {
        int p;
        int64_t e0;
        elems(grp, p, e0);
        mbar_arrive_expect_tx(&bar[s], BYTES);
        bulk_g2s(smem + s * STAGE, B.f[0][p] + e0 * NP3, BYTES, &bar[s]);
    };
    // the geometry factors of this thread's element in group grp (loaded one group ahead)
    auto geo = [&](int64_t grp) {
        int p;
        int64_t e0;
        const int ne = elems(grp, p, e0);
        return B.g[p][e0 + (el < ne ? el : 0)];
    };
    // per stage s: bit s of `phase` is its mbarrier parity, bit s of `pending` a copy in flight
    uint32_t phase = 0u;
    uint32_t pending = (full(blockIdx.x) ? 1u : 0u) | (full((int64_t)blockIdx.x + gridDim.x) ? 2u : 0u);
    if (tid == 0) {
        if (pending & 1u) issue(blockIdx.x, 0);
        if (pending & 2u) issue((int64_t)blockIdx.x + gridDim.x, 1);
    }
    float4 g_next = blockIdx.x < ngroups ? geo(blockIdx.x) : make_float4(0.f, 0.f, 0.f, 0.f);

    int it = 0;
    for (int64_t grp = blockIdx.x; grp < ngroups; grp += gridDim.x, ++it) {
        const int s = C::BULK ? (it & 1) : 0;
        float *st = smem + s * STAGE;
        int p;
        int64_t e0;
        const int ne = elems(grp, p, e0);
        const float4 g = g_next;
        if (grp + gridDim.x < ngroups) g_next = geo(grp + gridDim.x);
        if (C::BULK && ne == EPB) {
            // a wait that ran out leaves the stage pending, so the abort path drains its copy
            if (mbar_wait_bounded(&bar[s], (phase >> s) & 1u, err, B.wait_limit)) {
                phase ^= 1u << s;
                pending &= ~(1u << s);
            } else {
                s_abort = 1;
            }
        } else {
            for (int64_t idx = tid; idx < (int64_t)ne * NP3; idx += blockDim.x) st[idx] = B.f[0][p][e0 * NP3 + idx];
            if (C::BULK) fence_proxy_async_cta();  // a later bulk copy may overwrite these stores
        }
        __syncthreads();
        if (s_abort) break;
        if (active && el < ne) {
            const float *U = st + el * NP3;
            const int64_t eb = (e0 + el) * NP3;
            float u[NP], d[NP];
            // r-line (k, j) = (a, b): d/dr at the nodes (i, b, a)
            load_row<NP>(U + l * NP, u);
            contract_line2<NP>(u, d);
#pragma unroll
            for (int i = 0; i < NP; ++i) d[i] *= g.x;
            store_line<NP>(B.o[0][p] + eb + l * NP, d);
            // s-line (k, i) = (a, b): d/ds at the nodes (b, j', a)
#pragma unroll
            for (int m = 0; m < NP; ++m) u[m] = U[(a * NP + m) * NP + b];
            contract_line2<NP>(u, d);
            float *o1 = B.o[1][p] + eb + a * NP * NP + b;
#pragma unroll
            for (int m = 0; m < NP; ++m) o1[m * NP] = d[m] * g.y;
            // t-line (j, i) = (a, b): d/dt at the nodes (b, a, k')
#pragma unroll
            for (int m = 0; m < NP; ++m) u[m] = U[(m * NP + a) * NP + b];
            contract_line2<NP>(u, d);
            float *o2 = B.o[2][p] + eb + l;
#pragma unroll
            for (int m = 0; m < NP; ++m) o2[m * NP * NP] = d[m] * g.z;
        }
        __syncthreads();  // the stage is read
        if (tid == 0 && full(grp + 2 * (int64_t)gridDim.x)) {
            issue(grp + 2 * (int64_t)gridDim.x, s);
            pending |= 1u << s;
        }
    }
    // on an abort, wait (bounded) for copies still in flight into this CTA's shared memory
    if (C::BULK && s_abort && tid == 0) {
        for (int s = 0; s < 2; ++s)
            if ((pending >> s) & 1u) mbar_wait_bounded(&bar[s], (phase >> s) & 1u, nullptr);
    }
}

// ------------------------------------------------------------------------------------------
// Q for the other orders with direction-owned lines (the scheme of k_sem_q8 below, for any
// NP).  A thread that contracts all three directions for its own r-line reads its whole slab
// and column, (2 NP + 1) NP values per component, and repeats the level shift of every s- and
// t-line it touches.  Here thread (el, l) of a stage, with (a, b) = (l / NP, l % NP), owns
// three lines of element el: the r-line (k, j) = (a, b), the s-line (k, i) = (a, b) and the
// t-line (j, i) = (a, b).  It reads NP values per line; the s- and t-line owners write their NP
// derivatives to exchange slots laid out like the element, [k][j][i] (three slots of their own
// and the stage's component-0 part once that is read), from which the r-line owner reads its
// node row of each and folds the six products of Q: five barriers per stage.  Every line is
// contracted by contract_line2 (level shift, then the products in m order), the folds come in
// the same order, so the result is the one-thread-per-r-line result bit for bit.
// ------------------------------------------------------------------------------------------
template <int NP>
__global__ void __launch_bounds__(QCfg<NP>::NT, QCfg<NP>::MINB) k_sem_qd(const __grid_constant__ GBatch B, int *err)
{
    using C = QCfg<NP>;
    constexpr int NP3 = C::NP3, L = C::L, EPB = C::EPB;
    constexpr int CS = EPB * NP3;  // one component of a stage
    constexpr int STAGE = 3 * CS;
    constexpr uint32_t BYTES = CS * 4;
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int s_abort;
    float *X = smem + C::NSTAGE * STAGE;  // exchange: three slots of one component's stage size

    const int tid = threadIdx.x;
    const bool active = tid < EPB * L;
    const int el = active ? tid / L : 0, l = tid % L, a = l / NP, b = l % NP;
    const int64_t ngroups = B.gstart[B.n];
    // group -> (partition, its elements): a full group (EPB elements) can come by bulk copy
    auto elems = [&](int64_t grp, int &p, int64_t &e0) {
        p = qb_find(B, grp);
        e0 = (grp - B.gstart[p]) * EPB;
        const int64_t left = B.E[p] - e0;
        return (int)(left < EPB ? left : EPB);
    };
    if (tid == 0) {
        s_abort = 0;
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();

    auto full = [&](int64_t grp) {
        int p;
        int64_t e0;
        return C::BULK && grp < ngroups && elems(grp, p, e0) == EPB;
    };
    auto issue = [&](int64_t grp, int s) {
        int p;
        int64_t e0;
        elems(grp, p, e0);
        float *dst = smem + s * STAGE;
        mbar_arrive_expect_tx(&bar[s], 3 * BYTES);
#pragma unroll
        for (int c = 0; c < 3; ++c) bulk_g2s(dst + c * CS, B.f[c][p] + e0 * NP3, BYTES, &bar[s]);
    };
    // the geometry factors of this thread's element in group grp (loaded one group ahead)
    auto geo = [&](int64_t grp) {
        int p;
        int64_t e0;
        const int ne = elems(grp, p, e0);
        return B.g[p][e0 + (el < ne ? el : 0)];
    };
    // per stage s: bit s of `phase` is its mbarrier parity, bit s of `pending` a copy in flight
    uint32_t phase = 0u;
    uint32_t pending = (full(blockIdx.x) ? 1u : 0u) | (full((int64_t)blockIdx.x + gridDim.x) ? 2u : 0u);
    if (tid == 0) {
        if (pending & 1u) issue(blockIdx.x, 0);
        if (pending & 2u) issue((int64_t)blockIdx.x + gridDim.x, 1);
    }
    float4 g_next = blockIdx.x < ngroups ? geo(blockIdx.x) : make_float4(0.f, 0.f, 0.f, 0.f);

    int it = 0;
    for (int64_t grp = blockIdx.x; grp < ngroups; grp += gridDim.x, ++it) {
        const int s = C::BULK ? (it & 1) : 0;
        float *st = smem + s * STAGE;
        int p;
        int64_t e0;
        const int ne = elems(grp, p, e0);
        const float4 g = g_next;
        if (grp + gridDim.x < ngroups) g_next = geo(grp + gridDim.x);
        if (C::BULK && ne == EPB) {
            // a wait that ran out leaves the stage pending, so the abort path drains its copy
            if (mbar_wait_bounded(&bar[s], (phase >> s) & 1u, err, B.wait_limit)) {
                phase ^= 1u << s;
                pending &= ~(1u << s);
            } else {
                s_abort = 1;
            }
        } else {
            for (int c = 0; c < 3; ++c)
                for (int64_t idx = tid; idx < (int64_t)ne * NP3; idx += blockDim.x)
                    st[c * CS + idx] = B.f[c][p][e0 * NP3 + idx];
        }
        __syncthreads();
        if (s_abort) break;
        // the other stage was read (fold included) before the barrier above: its next group
        if (C::BULK && tid == 0 && it > 0 && full(grp + gridDim.x)) {
            issue(grp + gridDim.x, s ^ 1);
            pending |= 2u >> s;
        }
        const int64_t e = e0 + el;
        // Q = -1/2 sum_ij J_ij J_ji, J_ij = g_j d_j(u_i): c = -1/2 g_i g_j (x2 off the diagonal)
        const float c11 = -0.5f * g.x * g.x, c22 = -0.5f * g.y * g.y, c33 = -0.5f * g.z * g.z;
        const float c12 = -g.x * g.y, c13 = -g.x * g.z, c23 = -g.y * g.z;
        // this thread's s- and t-lines of component c -> exchange slots xs and xt
        auto st_lines = [&](int c, float *xs, float *xt) {
            if (!active) return;
            const float *U = st + c * CS + el * NP3;
            float u[NP], d[NP];
#pragma unroll
            for (int m = 0; m < NP; ++m) u[m] = U[(a * NP + m) * NP + b];
            contract_line2<NP>(u, d);
#pragma unroll
            for (int m = 0; m < NP; ++m) xs[el * NP3 + (a * NP + m) * NP + b] = d[m];
#pragma unroll
            for (int m = 0; m < NP; ++m) u[m] = U[(m * NP + a) * NP + b];
            contract_line2<NP>(u, d);
#pragma unroll
            for (int m = 0; m < NP; ++m) xt[el * NP3 + (m * NP + a) * NP + b] = d[m];
        };
        auto r_line = [&](int c, float (&dr)[NP]) {
            float u[NP];
            load_row<NP>(st + c * CS + el * NP3 + l * NP, u);
            contract_line2<NP>(u, dr);
        };
        auto x_row = [&](const float *x, float (&v)[NP]) { load_row<NP>(x + el * NP3 + l * NP, v); };
        // exchange slots A, B, C, and D: component 0's part of the stage, free once it is read
        float *XA = X, *XB = X + CS, *XC = X + 2 * CS, *XD = st;
        // the six products, each folded in as soon as its second factor is known
        float q[NP], dr[NP], x0[NP], x1[NP];
        st_lines(0, XA, XB);  // u_s -> A, u_t -> B
        if (active) {
            r_line(0, dr);
#pragma unroll
            for (int i = 0; i < NP; ++i) q[i] = c11 * dr[i] * dr[i];
        }
        __syncthreads();      // component 0 is read: D is free
        st_lines(1, XC, XD);  // v_s -> C, v_t -> D
        if (active) r_line(1, dr);
        __syncthreads();
        if (active) {
            x_row(XA, x0);  // u_s
            x_row(XC, x1);  // v_s
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                q[i] = fmaf(c12 * x0[i], dr[i], q[i]);
                q[i] = fmaf(c22 * x1[i], x1[i], q[i]);
            }
        }
        __syncthreads();      // A and C are free
        st_lines(2, XA, XC);  // w_s -> A, w_t -> C
        if (active) r_line(2, dr);
        __syncthreads();
        if (active) {
            x_row(XB, x0);  // u_t
#pragma unroll
            for (int i = 0; i < NP; ++i) q[i] = fmaf(c13 * x0[i], dr[i], q[i]);
            x_row(XD, x0);  // v_t
            x_row(XA, x1);  // w_s
#pragma unroll
            for (int i = 0; i < NP; ++i) q[i] = fmaf(c23 * x0[i], x1[i], q[i]);
            x_row(XC, x0);  // w_t
#pragma unroll
            for (int i = 0; i < NP; ++i) q[i] = fmaf(c33 * x0[i], x0[i], q[i]);
            if (el < ne) store_line<NP>(B.o[0][p] + e * NP3 + l * NP, q);
        }
        if constexpr (C::BULK) {
            // D (and a group loaded without a copy) was written through the generic proxy; a bulk
            // copy overwrites the stage after the next barrier
            fence_proxy_async_cta();
        } else {
            __syncthreads();  // one stage: the next group's loads overwrite D, still read by the fold above
        }
    }
    // on an abort, wait (bounded) for copies still in flight into this CTA's shared memory
    if (C::BULK && s_abort && tid == 0) {
        for (int s = 0; s < 2; ++s)
            if ((pending >> s) & 1u) mbar_wait_bounded(&bar[s], (phase >> s) & 1u, nullptr);
    }
}

// ------------------------------------------------------------------------------------------
// Q for N = 7 with direction-owned lines.  In k_sem_grad every thread contracts along all
// three directions for its own r-line, so it reads its whole slab and column (128 values per
// component, mostly broadcast).  Here each direction is contracted by the threads that
// own its lines: warp w is the s-line owner of slab k = w (lanes: element el = lane/8, node
// i = lane%8) and the t-line owner of plane j = w; each reads 8 values with conflict-free
// 4-byte loads (elements sit 520 floats apart in shared memory, shifting their banks by 8) and
// passes its 8 derivatives through an exchange buffer to the r-line owner (el, k, j), which
// contracts its own row and folds the six products of Q in k_sem_qd's order.
// 4 elements per stage, 2 stages fed by per-element bulk copies; 3 CTAs per SM.
// ------------------------------------------------------------------------------------------
// All eight outputs of the contraction (D u)_i, N = 7, by the even/odd split above; the
// {E_i, O_i} pair is carried in one float2 (__ffma2_rn: two round-to-nearest FMAs per
// instruction on Blackwell's FP32 pipe).
__device__ __forceinline__ void deriv8_eo(const float (&u)[8], float (&out)[8])
{
    float2 eo[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) eo[m] = make_float2(u[m] + u[7 - m], u[m] - u[7 - m]);
    // the line's level shift: the even coefficients of a row sum to zero (D 1 = 0), so
    // subtracting e_0 from every even part leaves the result unchanged in exact arithmetic and
    // makes the rounding follow the field's variation along the line, not its magnitude
#pragma unroll
    for (int m = 1; m < 4; ++m) eo[m].x -= eo[0].x;
    eo[0].x = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float2 a = __ffma2_rn(c_Deo7[i * 4 + 0], eo[0], make_float2(0.f, 0.f));
        a = __ffma2_rn(c_Deo7[i * 4 + 1], eo[1], a);
        a = __ffma2_rn(c_Deo7[i * 4 + 2], eo[2], a);
        a = __ffma2_rn(c_Deo7[i * 4 + 3], eo[3], a);
        out[i] = a.x + a.y;
        out[7 - i] = a.y - a.x;
    }
}

namespace q8 {
constexpr int EPB = 4, NP3 = 512, ES = 520;              // elements per stage, padded element stride
constexpr int CS = EPB * ES;                              // one component of a stage
constexpr int STAGE = 3 * CS;                             // floats per stage
constexpr int XS = 2 * CS;                                // exchange: s then t derivatives
constexpr size_t SMEM = sizeof(float) * (2 * STAGE + XS);
}  // namespace q8

// Triangle counts of one stage's elements from their node-row inside-bits (COUNT = true):
// rows[q][el][k * 8 + j] holds bit i = [Q(i, j, k) >= iso_q].  Thread (el, k, j) classifies the
// cut cells of row pair (j, k) (j, k < 7) as the isosurface pass does, each warp sums its half of
// the element, and part[q][el][half] receives the sums (their total is the element's count: the
// same as the counting pass of sem_isosurface_multi on the stored Q, bit-exact, as the same FP32
// values meet the same isovalues).
__device__ __forceinline__ void q8_count_stage(const GBatch &B, const uint8_t (*rows)[q8::EPB][64],
                                               int (*part)[q8::EPB][2], const uint8_t *s_nt, int ne, int el,
                                               int k, int j, int warp, int lane)
{
    for (int q = 0; q < B.niso; ++q) {
        int acc = 0;
        if (el < ne && j < 7 && k < 7) {
            const uint8_t *r = rows[q][el];
            const uint32_t r00 = r[k * 8 + j], r01 = r[k * 8 + j + 1], r10 = r[k * 8 + 8 + j], r11 = r[k * 8 + 9 + j];
            const uint32_t A = r00 & r01 & r10 & r11, O = r00 | r01 | r10 | r11;
            for (uint32_t act = (O | (O >> 1)) & ~(A & (A >> 1)) & 0x7Fu; act; act &= act - 1u) {
                const int i = __ffs(act) - 1;
                const int cs = (int)(((r00 >> i) & 3u) | (((r01 >> i) & 3u) << 2) | (((r10 >> i) & 3u) << 4) |
                                     (((r11 >> i) & 3u) << 6));
                acc += s_nt[cs];
            }
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
        if (lane == 0) part[q][el][warp & 1] = acc;
    }
}

// The counts of the stage before (its sums are complete after a barrier): cnt[q E + e0 + el].
__device__ __forceinline__ void q8_count_write(const GBatch &B, const int (*part)[q8::EPB][2], int64_t e0, int ne,
                                               int tid)
{
    const int q = tid / q8::EPB, el = tid % q8::EPB;
    if (q < B.niso && el < ne) B.cnt[(int64_t)q * B.E[0] + e0 + el] = part[q][el][0] + part[q][el][1];
}

template <bool COUNT>
__global__ void __launch_bounds__(256, 3) k_sem_q8(const __grid_constant__ GBatch B, int *err)
{
    using namespace q8;
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int s_abort;
    // COUNT: the stage's node-row inside-bits per isovalue, and the case table's triangle counts
    __shared__ uint8_t s_rows[COUNT ? SEM_MAX_ISO : 1][EPB][64];
    __shared__ int s_part[COUNT ? SEM_MAX_ISO : 1][EPB][2];
    __shared__ uint8_t s_nt[COUNT ? 256 : 1];
    if constexpr (COUNT)
        for (int t = threadIdx.x; t < 256; t += blockDim.x) s_nt[t] = B.ntri[t];
    float *X = smem + 2 * STAGE;  // exchange buffer
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // r-line owner (el, k, j)
    const int el = tid >> 6, k = (tid >> 3) & 7, j = tid & 7;
    // s-/t-line owner: element lane/8, node i = lane%8, slab k = warp (s), plane j = warp (t)
    const int oe = lane >> 3, oi = lane & 7;
    const int64_t ngroups = B.gstart[B.n];
    // group -> (partition, its elements): a full group (EPB elements) comes by bulk copies
    auto elems = [&](int64_t grp, int &p, int64_t &e0) {
        p = qb_find(B, grp);
        e0 = (grp - B.gstart[p]) * EPB;
        const int64_t left = B.E[p] - e0;
        return (int)(left < EPB ? left : EPB);
    };
    auto full = [&](int64_t grp) {
        int p;
        int64_t e0;
        return grp < ngroups && elems(grp, p, e0) == EPB;
    };
    if (tid == 0) {
        s_abort = 0;
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int64_t grp, int s) {
        int p;
        int64_t e0;
        elems(grp, p, e0);
        float *dst = smem + s * STAGE;
        mbar_arrive_expect_tx(&bar[s], 3 * EPB * NP3 * 4);
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int e = 0; e < EPB; ++e)
                bulk_g2s(dst + c * CS + e * ES, B.f[c][p] + (e0 + e) * NP3, NP3 * 4, &bar[s]);
    };
    // per stage s: bit s of `phase` is its mbarrier parity, bit s of `pending` a copy in flight
    uint32_t phase = 0u;
    uint32_t pending = (full(blockIdx.x) ? 1u : 0u) | (full((int64_t)blockIdx.x + gridDim.x) ? 2u : 0u);
    if (tid == 0) {
        if (pending & 1u) issue(blockIdx.x, 0);
        if (pending & 2u) issue(blockIdx.x + gridDim.x, 1);
    }
    const int sw = (j >> 2) & 1;  // row chunk stagger: j = 0..3 and 4..7 hit different banks
    int it = 0;
    for (int64_t grp = blockIdx.x; grp < ngroups; grp += gridDim.x, ++it) {
        const int s = it & 1;
        float *st = smem + s * STAGE;
        int p;
        int64_t e0;
        const int ne = elems(grp, p, e0);
        if (ne == EPB) {
            // a wait that ran out leaves the stage pending, so the abort path drains its copy
            if (mbar_wait_bounded(&bar[s], (phase >> s) & 1u, err, B.wait_limit)) {
                phase ^= 1u << s;
                pending &= ~(1u << s);
            } else {
                s_abort = 1;
            }
        } else {
            for (int c = 0; c < 3; ++c)
                for (int idx = tid; idx < ne * NP3; idx += 256)
                    st[c * CS + (idx / NP3) * ES + idx % NP3] = B.f[c][p][e0 * NP3 + idx];
            fence_proxy_async_cta();  // a later bulk copy may overwrite these stores
        }
        __syncthreads();
        if (s_abort) break;
        if constexpr (COUNT)
            if (it > 0) {  // the previous stage's sums are complete
                int pp;
                int64_t pe0;
                const int pne = elems(grp - gridDim.x, pp, pe0);
                q8_count_write(B, s_part, pe0, pne, tid);
            }
        const int64_t e = e0 + el;
        const float4 g = B.g[p][el < ne ? e : e0];
        const float c11 = -0.5f * g.x * g.x, c22 = -0.5f * g.y * g.y, c33 = -0.5f * g.z * g.z;
        const float c12 = -g.x * g.y, c13 = -g.x * g.z, c23 = -g.y * g.z;
        float q[8], su[8], tu[8], tv[8];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float *U = st + c * CS;
            // s-lines of slab `warp`: d/ds at nodes (i, j', k) for j' = 0..7
            {
                float u[8], d[8];
#pragma unroll
                for (int m = 0; m < 8; ++m) u[m] = U[oe * ES + (warp * 8 + m) * 8 + oi];
                deriv8_eo(u, d);
                // exchange rows (k, j) hold node i at position i ^ (j & 4): rows j = 0..3 and 4..7
                // keep their halves in swapped places, so the row owners' 16-byte reads below are
                // conflict-free in node order
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) X[oe * ES + (warp * 8 + jj) * 8 + (oi ^ (jj & 4))] = d[jj];
            }
            // t-lines of plane `warp`: d/dt at nodes (i, j, k') for k' = 0..7
            {
                float u[8], d[8];
#pragma unroll
                for (int m = 0; m < 8; ++m) u[m] = U[oe * ES + (m * 8 + warp) * 8 + oi];
                deriv8_eo(u, d);
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) X[CS + oe * ES + (kk * 8 + warp) * 8 + (oi ^ (warp & 4))] = d[kk];
            }
            // r-line of the owner (el, k, j)
            float dr[8];
            {
                const float4 *rp = reinterpret_cast<const float4 *>(U + el * ES + (k * 8 + j) * 8);
                const float4 A = rp[sw], B = rp[sw ^ 1];
                const float4 lo = sw ? B : A, hi = sw ? A : B;
                const float row[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
                deriv8_eo(row, dr);
            }
            __syncthreads();  // the exchange holds this component's s and t derivatives
            float ds[8], dt[8];
            {
                // the swizzled rows: nodes 0..3 sit in half sw, nodes 4..7 in half sw ^ 1
                const float4 *sp = reinterpret_cast<const float4 *>(X + el * ES + (k * 8 + j) * 8);
                const float4 *tp = reinterpret_cast<const float4 *>(X + CS + el * ES + (k * 8 + j) * 8);
                const float4 slo = sp[sw], shi = sp[sw ^ 1], tlo = tp[sw], thi = tp[sw ^ 1];
                ds[0] = slo.x; ds[1] = slo.y; ds[2] = slo.z; ds[3] = slo.w;
                ds[4] = shi.x; ds[5] = shi.y; ds[6] = shi.z; ds[7] = shi.w;
                dt[0] = tlo.x; dt[1] = tlo.y; dt[2] = tlo.z; dt[3] = tlo.w;
                dt[4] = thi.x; dt[5] = thi.y; dt[6] = thi.z; dt[7] = thi.w;
            }
            // Q = -1/2 sum_ij J_ij J_ji, J_ij = g_j d_j(u_i): the six products in k_sem_qd's order
            if (c == 0) {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    q[i] = c11 * dr[i] * dr[i];
                    su[i] = ds[i];
                    tu[i] = dt[i];
                }
            } else if (c == 1) {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    q[i] = fmaf(c12 * su[i], dr[i], q[i]);
                    q[i] = fmaf(c22 * ds[i], ds[i], q[i]);
                    tv[i] = dt[i];
                }
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    q[i] = fmaf(c13 * tu[i], dr[i], q[i]);
                    q[i] = fmaf(c23 * tv[i], ds[i], q[i]);
                    q[i] = fmaf(c33 * dt[i], dt[i], q[i]);
                }
                if constexpr (COUNT)  // the row's inside-bits, complete for the stage at the barrier below
                    for (int qi = 0; qi < B.niso; ++qi) {
                        uint32_t bits = 0;
#pragma unroll
                        for (int i = 0; i < 8; ++i) bits |= (q[i] >= B.iso[qi] ? 1u : 0u) << i;
                        s_rows[qi][el][k * 8 + j] = (uint8_t)bits;
                    }
            }
            __syncthreads();  // the exchange is free for the next component
        }

        if (el < ne) store_line<8>(B.o[0][p] + e * NP3 + (k * 8 + j) * 8, q);
        if (tid == 0 && full(grp + 2 * (int64_t)gridDim.x)) {
            issue(grp + 2 * gridDim.x, s);
            pending |= 1u << s;
        }
        // after the copy two stages ahead is on its way: the stage's triangle counts
        if constexpr (COUNT) q8_count_stage(B, s_rows, s_part, s_nt, ne, el, k, j, warp, lane);
    }
    if (s_abort && tid == 0) {
        for (int s = 0; s < 2; ++s)
            if ((pending >> s) & 1u) mbar_wait_bounded(&bar[s], (phase >> s) & 1u, nullptr);
    }
    if constexpr (COUNT) {
        // the last stage's counts (s_abort is uniform: every thread has seen the same value)
        __syncthreads();
        if (!s_abort && it > 0) {
            int pp;
            int64_t pe0;
            const int pne = elems((int64_t)blockIdx.x + (int64_t)(it - 1) * gridDim.x, pp, pe0);
            q8_count_write(B, s_part, pe0, pne, tid);
        }
    }
}

// A batch table for partitions [first, first + n) of (meshes, fields); EPB elements per group.
static void fill_batch(GBatch &B, int n, int epb, const sem_mesh *const *m, const float *const *f0,
                       const float *const *f1, const float *const *f2, float *const *o0, float *const *o1,
                       float *const *o2)
{
    memset(&B, 0, sizeof B);
    B.n = n;
    int64_t g = 0;
    for (int p = 0; p < n; ++p) {
        B.gstart[p] = g;
        B.E[p] = m[p]->E;
        B.f[0][p] = f0[p];
        B.f[1][p] = f1 ? f1[p] : nullptr;
        B.f[2][p] = f2 ? f2[p] : nullptr;
        B.o[0][p] = o0[p];
        B.o[1][p] = o1 ? o1[p] : nullptr;
        B.o[2][p] = o2 ? o2[p] : nullptr;
        B.g[p] = m[p]->g;
        g += (m[p]->E + epb - 1) / epb;
    }
    B.gstart[n] = g;
}

// Candidate launch widths of a persistent Q kernel: 1 .. max_per_sm resident CTAs per SM (the
// elements each CTA walks through scale inversely), the widest first
static int q_width_candidates(int max_per_sm, int *cand)
{
    int n = 0;
    for (int w = max_per_sm; w >= 1 && n < 4; --w) cand[n++] = w;
    return n;
}

template <bool COUNT>
static sem_status launch_q8(sem_ctx *ctx, const GBatch &B)
{
    static KernelSetup ks;  // per instantiation and device
    int per_sm = 1;
    SEM_TRY(kernel_setup(ctx, ks, k_sem_q8<COUNT>, 256, q8::SMEM, &per_sm));
    const int64_t ngroups = B.gstart[B.n];
    if (ngroups == 0) return SEM_OK;
    int cand[4];
    const int nc = q_width_candidates(per_sm, cand);
    int64_t E = 0;
    for (int p = 0; p < B.n; ++p) E += B.E[p];
    return width_tuned(ctx, COUNT ? TUNE_Q8_COUNT : TUNE_Q8, 7, E, cand, nc, per_sm, [&](int w) -> sem_status {
        int64_t grid = (int64_t)ctx->sm_count * w;
        if (grid > ngroups) grid = ngroups;
        SEM_TRACED(ctx, COUNT ? "k_sem_q8_count" : "k_sem_q8",
                   k_sem_q8<COUNT><<<(unsigned)grid, 256, q8::SMEM, ctx->stream>>>(B, ctx->d_flag));
        return sem_cuda(ctx, cudaGetLastError(), "k_sem_q8 launch");
    });
}

template <int NP>
static sem_status launch_grad(sem_ctx *ctx, const GBatch &B)
{
    using C = QCfg<NP>;
    const size_t smem = sizeof(float) * (size_t)C::NSTAGE * C::EPB * C::NP3;
    auto kern = k_sem_grad<NP>;
    static KernelSetup ks;  // per instantiation and device
    int per_sm = 1;
    SEM_TRY(kernel_setup(ctx, ks, kern, C::NT, smem, &per_sm));
    const int64_t ngroups = B.gstart[B.n];
    if (ngroups == 0) return SEM_OK;
    int cand[4];
    const int nc = q_width_candidates(per_sm, cand);
    int64_t E = 0;
    for (int p = 0; p < B.n; ++p) E += B.E[p];
    return width_tuned(ctx, TUNE_QGRAD_DERIV, NP - 1, E, cand, nc, per_sm,
                       [&](int w) -> sem_status {
                           int64_t grid = (int64_t)ctx->sm_count * w;
                           if (grid > ngroups) grid = ngroups;
                           SEM_TRACED(ctx, "k_sem_grad",
                                      kern<<<(unsigned)grid, C::NT, smem, ctx->stream>>>(B, ctx->d_flag));
                           return sem_cuda(ctx, cudaGetLastError(), "k_sem_grad launch");
                       });
}

// Q of the other orders: two stages of the three components and the exchange's three slots
template <int NP>
static sem_status launch_qd(sem_ctx *ctx, const GBatch &B)
{
    using C = QCfg<NP>;
    const size_t smem = sizeof(float) * (size_t)(C::NSTAGE * 3 + 3) * C::EPB * C::NP3;
    auto kern = k_sem_qd<NP>;
    static KernelSetup ks;  // per instantiation and device
    int per_sm = 1;
    SEM_TRY(kernel_setup(ctx, ks, kern, C::NT, smem, &per_sm));
    const int64_t ngroups = B.gstart[B.n];
    if (ngroups == 0) return SEM_OK;
    int cand[4];
    const int nc = q_width_candidates(per_sm, cand);
    int64_t E = 0;
    for (int p = 0; p < B.n; ++p) E += B.E[p];
    return width_tuned(ctx, TUNE_QGRAD, NP - 1, E, cand, nc, per_sm, [&](int w) -> sem_status {
        int64_t grid = (int64_t)ctx->sm_count * w;
        if (grid > ngroups) grid = ngroups;
        SEM_TRACED(ctx, "k_sem_qd", kern<<<(unsigned)grid, C::NT, smem, ctx->stream>>>(B, ctx->d_flag));
        return sem_cuda(ctx, cudaGetLastError(), "k_sem_qd launch");
    });
}

template <int NC>
static sem_status dispatch(sem_ctx *ctx, int N, int n, const sem_mesh *const *m, const float *const *f0,
                           const float *const *f1, const float *const *f2, float *const *o0, float *const *o1,
                           float *const *o2)
{
    GBatch B;
    if (NC == 3 && N == 7) {
        fill_batch(B, n, q8::EPB, m, f0, f1, f2, o0, o1, o2);
        B.wait_limit = ctx->wait_limit;
        return launch_q8<false>(ctx, B);
    }
    switch (N + 1) {
#define SEM_CASE(NPV)                                                        \
    case NPV:                                                                \
        fill_batch(B, n, QCfg<NPV>::EPB, m, f0, f1, f2, o0, o1, o2);         \
        B.wait_limit = ctx->wait_limit;                                      \
        return NC == 3 ? launch_qd<NPV>(ctx, B) : launch_grad<NPV>(ctx, B);
        SEM_CASE(2) SEM_CASE(3) SEM_CASE(4) SEM_CASE(5) SEM_CASE(6) SEM_CASE(7) SEM_CASE(8) SEM_CASE(9)
        SEM_CASE(10) SEM_CASE(11) SEM_CASE(12) SEM_CASE(13) SEM_CASE(14) SEM_CASE(15) SEM_CASE(16)
#undef SEM_CASE
    default: return sem_fail(ctx, SEM_ERR_ARG, "order N=%d not supported", N);
    }
}

// ------------------------------------------------------------------------------------------
// General (curved) elements: the isoparametric chain rule at every node,
//   d u / d x_j = sum_d (d u / d r_d) (d r_d / d x_j),
// with the reference derivatives d u / d r_d = sum_m D[idx_d][m] u(idx_d -> m) and the inverse
// Jacobian d r_d / d x_j of each node precomputed by sem_load_mesh (plane 3 d + j of geo).
// A block takes one element at a time (grid-stride): its NC components and D in shared
// memory, one thread per node.  NC = 1: the three derivatives; NC = 3: Q = -1/2 sum_ij J_ij J_ji.
// ------------------------------------------------------------------------------------------
#define GEN_THREADS 256
template <int NP, int NC>
__global__ void __launch_bounds__(GEN_THREADS) k_sem_grad_gen(const float *__restrict__ f0, const float *__restrict__ f1,
                                                             const float *__restrict__ f2, const float *__restrict__ geo,
                                                             int64_t E, float *__restrict__ o0, float *__restrict__ o1,
                                                             float *__restrict__ o2)
{
    constexpr int NP3 = NP * NP * NP;
    extern __shared__ float s_u[];  // NC * NP3
    __shared__ float s_D[NP * NP];
    for (int q = threadIdx.x; q < NP * NP; q += blockDim.x) s_D[q] = Dc<NP>(q / NP, q % NP);
    const int64_t tot = E * NP3;
    const float *src[3] = {f0, f1, f2};
    for (int64_t e = blockIdx.x; e < E; e += gridDim.x) {
        __syncthreads();  // the previous element's readers are done (and D is in place)
#pragma unroll
        for (int c = 0; c < NC; ++c)
            for (int n = threadIdx.x; n < NP3; n += blockDim.x) s_u[c * NP3 + n] = __ldg(src[c] + e * NP3 + n);
        __syncthreads();
        for (int n = threadIdx.x; n < NP3; n += blockDim.x) {
            const int i = n % NP, j = (n / NP) % NP, k = n / (NP * NP);
            const int64_t node = e * NP3 + n;
            float G[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) G[q] = __ldg(geo + q * tot + node);
            float J[NC][3];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const float *U = s_u + c * NP3;
                // each line shifted by its first value (D 1 = 0; see contract_line2)
                const float lr = U[(k * NP + j) * NP], ls = U[(k * NP) * NP + i], lt = U[j * NP + i];
                float dr = 0.f, ds = 0.f, dt = 0.f;
#pragma unroll
                for (int m = 1; m < NP; ++m) {
                    dr = fmaf(s_D[i * NP + m], U[(k * NP + j) * NP + m] - lr, dr);
                    ds = fmaf(s_D[j * NP + m], U[(k * NP + m) * NP + i] - ls, ds);
                    dt = fmaf(s_D[k * NP + m], U[(m * NP + j) * NP + i] - lt, dt);
                }
#pragma unroll
                for (int jj = 0; jj < 3; ++jj) J[c][jj] = fmaf(dt, G[6 + jj], fmaf(ds, G[3 + jj], dr * G[jj]));
            }
            if constexpr (NC == 1) {
                o0[node] = J[0][0];
                o1[node] = J[0][1];
                o2[node] = J[0][2];
            } else {
                const float d = fmaf(J[0][0], J[0][0], fmaf(J[1][1], J[1][1], J[2][2] * J[2][2]));
                const float o = fmaf(J[0][1], J[1][0], fmaf(J[0][2], J[2][0], J[1][2] * J[2][1]));
                o0[node] = -0.5f * fmaf(2.f, o, d);
            }
        }
    }
}

template <int NC>
static sem_status launch_gen(sem_ctx *ctx, const sem_mesh *m, const float *f0, const float *f1, const float *f2,
                             float *o0, float *o1, float *o2)
{
    switch (m->N + 1) {
#define SEM_CASE(NPV)                                                                                          \
    case NPV: {                                                                                                \
        auto kern = k_sem_grad_gen<NPV, NC>;                                                                   \
        const size_t smem = sizeof(float) * NC * NPV * NPV * NPV;                                              \
        static KernelSetup ks; /* per instantiation and device */                                             \
        SEM_TRY(kernel_setup(ctx, ks, kern, 0, smem));                                                         \
        const int64_t grid = std::min<int64_t>(m->E, (int64_t)ctx->sm_count * 8);                             \
        SEM_TRACED(ctx, "k_sem_grad_gen",                                                                      \
                   kern<<<(unsigned)grid, GEN_THREADS, smem, ctx->stream>>>(f0, f1, f2, m->geo, m->E, o0, o1, o2)); \
        return sem_cuda(ctx, cudaGetLastError(), "k_sem_grad_gen launch");                                    \
    }
        SEM_CASE(2) SEM_CASE(3) SEM_CASE(4) SEM_CASE(5) SEM_CASE(6) SEM_CASE(7) SEM_CASE(8) SEM_CASE(9)
        SEM_CASE(10) SEM_CASE(11) SEM_CASE(12) SEM_CASE(13) SEM_CASE(14) SEM_CASE(15) SEM_CASE(16)
#undef SEM_CASE
    default: return sem_fail(ctx, SEM_ERR_ARG, "order N=%d not supported", m->N);
    }
}

sem_status qcrit_count_launch(sem_ctx *ctx, const sem_mesh *m, const float *u, const float *v, const float *w,
                              float *Q, int niso, const float *isos, int32_t *cnt)
{
    GBatch B;
    fill_batch(B, 1, q8::EPB, &m, &u, &v, &w, &Q, nullptr, nullptr);
    B.wait_limit = ctx->wait_limit;
    B.niso = niso;
    for (int q = 0; q < niso; ++q) B.iso[q] = isos[q];
    B.cnt = cnt;
    B.ntri = ctx->d_ntri;
    return launch_q8<true>(ctx, B);
}

sem_status qcrit_launch(sem_ctx *ctx, const sem_mesh *m, const float *u, const float *v, const float *w, float *Q)
{
    if (m->curved) return launch_gen<3>(ctx, m, u, v, w, Q, nullptr, nullptr);
    return dispatch<3>(ctx, m->N, 1, &m, &u, &v, &w, &Q, nullptr, nullptr);
}

sem_status deriv_launch(sem_ctx *ctx, const sem_mesh *m, const float *u, float *dx, float *dy, float *dz)
{
    if (m->curved) return launch_gen<1>(ctx, m, u, nullptr, nullptr, dx, dy, dz);
    return dispatch<1>(ctx, m->N, 1, &m, &u, nullptr, nullptr, &dx, &dy, &dz);
}

// Q of several partitions: one persistent launch per order over all partitions of that order
// (at most QB_MAX per launch), in the order the partitions first appear.
sem_status qcrit_batch_launch(sem_ctx *ctx, int n, const sem_mesh *const *m, const float *const *u,
                              const float *const *v, const float *const *w, float *const *Q)
{
    std::vector<char> done(n, 0);
    std::vector<const sem_mesh *> mm;
    std::vector<const float *> uu, vv, ww;
    std::vector<float *> qq;
    for (int a = 0; a < n; ++a) {
        if (done[a]) continue;
        const int N = m[a]->N;
        mm.clear(), uu.clear(), vv.clear(), ww.clear(), qq.clear();
        for (int b = a; b < n; ++b)
            if (!done[b] && m[b]->N == N && m[b]->E > 0) {
                done[b] = 1;
                mm.push_back(m[b]), uu.push_back(u[b]), vv.push_back(v[b]), ww.push_back(w[b]), qq.push_back(Q[b]);
            }
        for (size_t c0 = 0; c0 < mm.size(); c0 += QB_MAX) {
            const int k = (int)std::min<size_t>(QB_MAX, mm.size() - c0);
            SEM_TRY(dispatch<3>(ctx, N, k, mm.data() + c0, uu.data() + c0, vv.data() + c0, ww.data() + c0,
                                qq.data() + c0, nullptr, nullptr));
        }
    }
    return SEM_OK;
}
