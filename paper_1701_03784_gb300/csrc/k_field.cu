// Field update of the mixed E-B leapfrog (Eqs. full_d_dfl, full_d_dal) and the per-step
// triangle field records read by the particle kernel.
#include <algorithm>

#include "pic_internal.h"

namespace pic {

// K3, one thread per face: B^{n+1/2} = B^{n-1/2} - dt (D_curl E^n)_f, and the record's
// field coefficients: E(lambda) = sum_k E_k (lambda_a grad lambda_b - lambda_b grad
// lambda_a) = sum_m lambda_m c_m (E_k plus the static field's edge value when one is set:
// it drives the particles but takes no part in the leapfrog), and
// B_phi = (B^{n+1/2} + B^{n-1/2}) / (2A) (W2 = 1/A).  In a lossy layer
// B^{n+1/2} = a_f B^{n-1/2} - b_f dt (D_curl E^n)_f.
// The same launch clears the step's accumulators (J per edge, Q_abs per node, and in the
// FP64 build Q^{n+1}, which the particle kernel accumulates).
template <class P, bool STATIC, bool LOSS>
__global__ void __launch_bounds__(512) k_field_b(FieldArgs<P> a) {
    using R = typename P::R;
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f < a.N1) a.J[f] = 0;
    if (f < a.N0) {
        a.Qabs[f] = 0;
        if constexpr (!P::fixed) a.Qnext[f] = 0;
    }
    if (f >= a.N2) return;
    if constexpr (sizeof(R) == 4) {
        // FP32 record: 16-byte groups (g | rho, 1/A | c0 c1 | c2, B_phi, pad | nodes, flags |
        // edges, flags), read and written as vectors
        float4 *R4 = reinterpret_cast<float4 *>(a.rec + f);
        const float4 G = R4[0], RH = R4[1];
        const int4 EG = reinterpret_cast<const int4 *>(a.rec + f)[5];
        const float g[3][2] = {{G.x, G.y}, {G.z, G.w}, {-G.x - G.z, -G.y - G.w}};
        float c[3][2] = {{0, 0}, {0, 0}, {0, 0}};
        float curl = 0;
        const int ek[3] = {EG.x, EG.y, EG.z};
        float E3[3], S3[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 3; k++) E3[k] = a.E[ek[k]];
        if constexpr (STATIC) {
#pragma unroll
            for (int k = 0; k < 3; k++) S3[k] = a.Es[ek[k]];
        }
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const float Ek = STATIC ? E3[k] + S3[k] : E3[k];   // the gather sees the static field
            const int i = (k + 1) % 3, j = (k + 2) % 3;
            const bool fwd = (EG.w >> k) & 1;
            const int ta = fwd ? i : j, hb = fwd ? j : i;
            c[ta][0] += Ek * g[hb][0];
            c[ta][1] += Ek * g[hb][1];
            c[hb][0] -= Ek * g[ta][0];
            c[hb][1] -= Ek * g[ta][1];
            curl += fwd ? E3[k] : -E3[k];
        }
        const float Bold = a.B[f];
        float Bnew = Bold - a.dt * curl;
        if constexpr (LOSS) {
            const float2 lf = reinterpret_cast<const float2 *>(a.loss_f)[f];
            Bnew = lf.x * Bold - lf.y * (a.dt * curl);
        }
        a.B[f] = Bnew;
        R4[2] = make_float4(c[0][0], c[0][1], c[1][0], c[1][1]);
        R4[3] = make_float4(c[2][0], c[2][1], 0.5f * (Bnew + Bold) * RH.w, 0.f);
        return;
    }
    TriRec<R> &rc = a.rec[f];
    const int32_t flags = rc.flags;
    R g[3][2] = {{rc.g[0], rc.g[1]}, {rc.g[2], rc.g[3]}, {-rc.g[0] - rc.g[2], -rc.g[1] - rc.g[3]}};
    R c[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    R curl = 0;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const R Ed = a.E[rc.edge[k]];
        R Ek = Ed;
        if constexpr (STATIC) Ek += a.Es[rc.edge[k]];   // the gather sees the static field
        int i = (k + 1) % 3, j = (k + 2) % 3;
        bool fwd = (flags >> k) & 1;   // edge runs (k+1) -> (k+2): D_curl entry +1
        int ta = fwd ? i : j, hb = fwd ? j : i;
        c[ta][0] += Ek * g[hb][0];
        c[ta][1] += Ek * g[hb][1];
        c[hb][0] -= Ek * g[ta][0];
        c[hb][1] -= Ek * g[ta][1];
        curl += fwd ? Ed : -Ed;
    }
    R Bold = a.B[f];
    R Bnew = Bold - a.dt * curl;
    if constexpr (LOSS) Bnew = a.loss_f[2 * f] * Bold - a.loss_f[2 * f + 1] * (a.dt * curl);
    a.B[f] = Bnew;
    rc.bphi = R(0.5) * (Bnew + Bold) * rc.inv_area;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        rc.c[2 * k] = c[k][0];
        rc.c[2 * k + 1] = c[k][1];
    }
}

// Per node, after the particle step.  FP32 build: Q^{n+1} = Q^n - (D_div J)/2^22 -
// Q_absorbed.  Per particle, the segment currents at a node sum to 2^22 (lambda^start -
// lambda^end) in the fixed-point units (the identity behind Eq. DCE), so D_div J is
// divisible by 2^22 and the result equals Eq. charge evaluated at the new positions
// exactly; a non-zero remainder would be a broken invariant and is counted.  Both builds:
// the charge removed at walls is summed since the Gauss-law reference.
template <class P>
__device__ __forceinline__ void node_update(const FieldArgs<P> &a, int64_t k) {
    if constexpr (P::fixed) {
        long long div = 0;
        for (int64_t q = a.node_ptr[k]; q < a.node_ptr[k + 1]; q++)
            div += (long long)a.node_sign[q] * (long long)a.J[a.node_edge[q]];
        if (div & (long long)(LAM_ONE - 1)) atomicAdd(a.counters + CNT_REMAINDER, 1ULL);
        long long qn = (long long)a.Qn[k] - (div >> LAM_BITS) - (long long)a.Qabs[k];
        a.Qnext[k] = (unsigned long long)qn;
    }
    a.Qwall[k] += a.Qabs[k];
}

// K4a, one thread per free edge: r = D_curl^T star_mu^-1 B^{n+1/2} - J^{n+1/2}; the DGL
// auxiliary flux D += dt r.  The same launch does the per-node update (thread k, node k).
template <class P>
__global__ void __launch_bounds__(512) k_field_r(FieldArgs<P> a) {
    using R = typename P::R;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.N0) node_update<P>(a, i);
    if (i >= a.nf) return;
    const int32_t e = a.free_edges[i];
    const int2 ef = reinterpret_cast<const int2 *>(a.edge_face)[i];
    double r = 0;
#pragma unroll
    for (int q = 0; q < 2; q++) {
        int32_t fs = q == 0 ? ef.x : ef.y;
        if (fs == 0) continue;
        int32_t f = (fs > 0 ? fs : -fs) - 1;
        double hf = (double)a.mu_inv[f] * (double)a.B[f];
        r += fs > 0 ? hf : -hf;
    }
    double Jp;
    if constexpr (P::fixed) Jp = (double)(long long)a.J[e] * a.j_scale;
    else Jp = a.J[e] * a.j_scale;
    r -= Jp;
    a.D[e] += (double)a.dt * r;
    a.r[i] = (R)r;
}

// K4b, sliced ELL SpMV over free edges: E_e += dt (M r)_i (in a lossy layer
// E_e <- a_e E_e + b_e dt (M r)_i, a = (1 - s)/(1 + s), b = 1/(1 + s), s = sigma dt/(2 eps0)).  A warp owns a slice of 32 rows
// stored column-major, so each step of the row loop reads 32 consecutive values.
template <class P, bool LOSS>
__global__ void __launch_bounds__(512) k_field_spmv(FieldArgs<P> a) {
    using R = typename P::R;
    int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t slice = row >> 5;
    int lane = (int)(row & 31);
    int64_t n_slices = (a.nf + 31) >> 5;
    if (slice >= n_slices) return;
    int64_t off = a.ell_off[slice];
    int width = (int)((a.ell_off[slice + 1] - off) >> 5);
    R acc = 0;
    int k = 0;
    // four columns' indices and values in flight before their gathers (the sum keeps the
    // column order)
    for (; k + 4 <= width; k += 4) {
        int32_t col[4];
        R val[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int64_t idx = off + ((int64_t)(k + u) << 5) + lane;
            col[u] = a.ell_col[idx];
            val[u] = a.ell_val[idx];
        }
        R rv[4];
#pragma unroll
        for (int u = 0; u < 4; u++) rv[u] = a.r[col[u]];
#pragma unroll
        for (int u = 0; u < 4; u++) acc += val[u] * rv[u];
    }
    for (; k < width; k++) {
        const int64_t idx = off + ((int64_t)k << 5) + lane;
        acc += a.ell_val[idx] * a.r[a.ell_col[idx]];
    }
    if (row < a.nf) {
        const int32_t e = a.free_edges[row];
        if constexpr (LOSS) a.E[e] = a.loss_e[2 * row] * a.E[e] + a.loss_e[2 * row + 1] * (a.dt * acc);
        else a.E[e] += a.dt * acc;
    }
}

template <class P>
void launch_field_b(const FieldArgs<P> &a, cudaStream_t s) {
    const int64_t n = std::max(a.N2, std::max(a.N1, a.N0));
    const int b = a.block;
    const unsigned g = (unsigned)((n + b - 1) / b);
    // the optional static field and lossy layer as instantiations: none costs the common
    // case anything
    if (a.Es && a.loss_f) k_field_b<P, true, true><<<g, b, 0, s>>>(a);
    else if (a.Es) k_field_b<P, true, false><<<g, b, 0, s>>>(a);
    else if (a.loss_f) k_field_b<P, false, true><<<g, b, 0, s>>>(a);
    else k_field_b<P, false, false><<<g, b, 0, s>>>(a);
    PIC_LAUNCHED();
}

template <class P>
void launch_field_e(const FieldArgs<P> &a, cudaStream_t s) {
    const int64_t n = std::max(a.nf, a.N0);
    const int b = a.block;
    k_field_r<P><<<(unsigned)((n + b - 1) / b), b, 0, s>>>(a);
    PIC_LAUNCHED();
    int64_t rows = ((a.nf + 31) / 32) * 32;
    if (a.loss_e) k_field_spmv<P, true><<<(unsigned)((rows + b - 1) / b), b, 0, s>>>(a);
    else k_field_spmv<P, false><<<(unsigned)((rows + b - 1) / b), b, 0, s>>>(a);
    PIC_LAUNCHED();
}

template void launch_field_b<PF32>(const FieldArgs<PF32> &, cudaStream_t);
template void launch_field_b<PF64>(const FieldArgs<PF64> &, cudaStream_t);
template void launch_field_e<PF32>(const FieldArgs<PF32> &, cudaStream_t);
template void launch_field_e<PF64>(const FieldArgs<PF64> &, cudaStream_t);

}  // namespace pic
