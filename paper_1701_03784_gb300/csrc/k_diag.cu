// K5: diagnostics (Sec. 3.5, Sec. 5.1.1) as FP64 reductions on the device, and read-back
// conversions.  Not on the per-step path.
#include <algorithm>
#include <type_traits>

#include "pic_internal.h"

namespace pic {

namespace {

__device__ __forceinline__ void atomic_max_pos(double *p, double v) {
    // non-negative doubles order like their bit patterns
    if (v > 0.0) atomicMax(reinterpret_cast<unsigned long long *>(p), __double_as_longlong(v));
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

}  // namespace

// Per node: DCE residual (Eq. DCE with the absorbed-charge sink), NR_DCE, DGL residual
// against its reference (Eq. DGL_RSD_REL) and max |Q|.
template <class P>
__global__ void __launch_bounds__(256) k_diag_nodes(DiagDev d, const typename P::Acc *J,
                                                    const typename P::Acc *Qn,
                                                    const typename P::Acc *Qp,
                                                    const typename P::Acc *Qabs,
                                                    const typename P::Acc *Qpos,
                                                    const typename P::Acc *Qwall, const double *D,
                                                    double *dgl_ref, int set_ref, double q_scale,
                                                    double *out) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double dce = 0, nr = 0, dgl = 0, qmax = 0, nz = 0;
    if (k < d.N0) {
        double qk;
        if constexpr (P::fixed) {
            long long div = 0;
            for (int64_t q = d.node_ptr[k]; q < d.node_ptr[k + 1]; q++)
                div += (long long)d.node_sign[q] * (long long)J[d.node_edge[q]];
            long long dq = (long long)Qn[k] - (long long)Qp[k] + (long long)Qabs[k];
            long long res = dq * (long long)LAM_ONE + div;  // exact: units 2^-44 of q_src
            dce = fabs((double)res) * J_INV;
            nz = res != 0 ? 1.0 : 0.0;
            if (Qpos) {
                // the carried Q^{n+1} against Eq. charge evaluated at the positions
                long long mis = (long long)Qn[k] - (long long)Qpos[k];
                if (mis != 0) nz = 1.0;
                dce = fmax(dce, fabs((double)mis) * LAM_INV);
            }
            double divd = fabs((double)div) * J_INV;
            if (divd > 1e-9) nr = dce / divd;
            qk = (double)(long long)Qn[k] * LAM_INV;
        } else {
            double div = 0;
            for (int64_t q = d.node_ptr[k]; q < d.node_ptr[k + 1]; q++)
                div += (double)d.node_sign[q] * J[d.node_edge[q]];
            double res = (Qn[k] - Qp[k] + Qabs[k]) + div;
            dce = fabs(res);
            if (fabs(div) > 1e-9) nr = dce / fabs(div);
            qk = Qn[k];
        }
        qk *= q_scale;
        qmax = fabs(qk);
        if (!d.node_on_pec[k]) {
            double s = 0;
            for (int64_t q = d.node_ptr[k]; q < d.node_ptr[k + 1]; q++)
                s += (double)d.node_sign[q] * D[d.node_edge[q]];
            // charge removed at walls since the reference leaves Q without crossing an
            // edge: it shifts res by exactly that amount, which is taken out here
            double qw;
            if constexpr (P::fixed) qw = (double)(long long)Qwall[k] * LAM_INV * q_scale;
            else qw = Qwall[k] * q_scale;
            double res = s - qk - qw;
            if (set_ref) dgl_ref[k] = res;
            else dgl = fabs(res - dgl_ref[k]);
        }
    }
    if (set_ref) return;
    dce = warp_max(dce);
    nr = warp_max(nr);
    dgl = warp_max(dgl);
    qmax = warp_max(qmax);
    nz = warp_sum(nz);
    if ((threadIdx.x & 31) == 0) {
        atomic_max_pos(out + 0, dce);
        if (nz > 0) atomicAdd(out + 1, nz);
        atomic_max_pos(out + 2, nr);
        atomic_max_pos(out + 3, dgl);
        atomic_max_pos(out + 4, qmax);
    }
}

// 1/2 E.star_eps.E + 1/2 sum star_mu^-1 B^2
template <class P>
__global__ void __launch_bounds__(256) k_diag_energy(DiagDev d, const typename P::R *E,
                                                     const typename P::R *B,
                                                     const typename P::R *mu_inv, double *out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0;
    if (i < d.N1) {
        double a = 0;
        for (int64_t q = d.eps_ptr[i]; q < d.eps_ptr[i + 1]; q++)
            a += d.eps_val[q] * (double)E[d.eps_idx[q]];
        s += 0.5 * a * (double)E[i];
    }
    if (i < d.N2) s += 0.5 * (double)mu_inv[i] * (double)B[i] * (double)B[i];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(out + 5, s);
}

// sum of (gamma - 1) over live particles; the FP32 build evaluates each term in FP32 (its
// momenta are FP32) and sums in FP64.  Grid-stride, one atomic per block.
template <class P>
__global__ void __launch_bounds__(256) k_diag_kinetic(Particles<P> p, const int64_t *n_slots,
                                                      double inv_c2, double *out) {
    __shared__ double part[8];
    const int64_t n = *n_slots;
    double s = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (p.tri[i] < 0) continue;
        if constexpr (P::fixed) {
            const float ic2 = (float)inv_c2;
            const float ur = p.ur[i], up = p.up[i], uz = p.uz[i];
            const float x = (ur * ur + up * up + uz * uz) * ic2;
            // (gamma - 1) without cancellation
            s += (double)(x / (sqrtf(1.f + x) + 1.f));
        } else {
            const double x = ((double)p.ur[i] * p.ur[i] + (double)p.up[i] * p.up[i] +
                              (double)p.uz[i] * p.uz[i]) * inv_c2;
            s += x / (sqrt(1.0 + x) + 1.0);
        }
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
        s = warp_sum(s);
        if (threadIdx.x == 0 && s != 0.0) atomicAdd(out + 6, s);
    }
}

template <class P>
void launch_diag(const DiagDev &d, const typename P::Acc *J, const typename P::Acc *Qn,
                 const typename P::Acc *Qp, const typename P::Acc *Qabs,
                 const typename P::Acc *Qpos, const typename P::Acc *Qwall, const double *D,
                 double *dgl_ref, int set_ref, const typename P::R *E, const typename P::R *B,
                 const typename P::R *mu_inv, Particles<P> p, const int64_t *n_slots,
                 int64_t n_bound, double q_scale, double inv_c2, double *out, cudaStream_t s) {
    k_diag_nodes<P><<<(unsigned)((d.N0 + 255) / 256), 256, 0, s>>>(d, J, Qn, Qp, Qabs, Qpos, Qwall, D, dgl_ref,
                                                                   set_ref, q_scale, out);
    PIC_LAUNCHED();
    if (set_ref) return;
    int64_t ne = d.N1 > d.N2 ? d.N1 : d.N2;
    k_diag_energy<P><<<(unsigned)((ne + 255) / 256), 256, 0, s>>>(d, E, B, mu_inv, out);
    PIC_LAUNCHED();
    if (n_bound > 0) {
        const int64_t blocks = std::min<int64_t>((n_bound + 255) / 256, 1216);
        k_diag_kinetic<P><<<(unsigned)blocks, 256, 0, s>>>(p, n_slots, inv_c2, out);
        PIC_LAUNCHED();
    }
}

template <class P>
__global__ void k_export(Particles<P> p, int64_t n, double *lam3, double *u3, int64_t *pid) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double l0, l1, l2;
    if constexpr (P::fixed) {
        int32_t a = p.l0[i], b = p.l1[i];
        l0 = a * LAM_INV;
        l1 = b * LAM_INV;
        l2 = (LAM_ONE - a - b) * LAM_INV;
    } else {
        l0 = p.l0[i];
        l1 = p.l1[i];
        l2 = 1.0 - l0 - l1;
    }
    lam3[3 * i] = l0;
    lam3[3 * i + 1] = l1;
    lam3[3 * i + 2] = l2;
    u3[3 * i] = p.ur[i];
    u3[3 * i + 1] = p.up[i];
    u3[3 * i + 2] = p.uz[i];
    pid[i] = p.pid[i];
}

template <class P>
void launch_export(Particles<P> p, int64_t n, const TriRec<typename P::R> *, double *lam3,
                   double *u3, int64_t *pid, cudaStream_t s) {
    if (n <= 0) return;
    k_export<P><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, n, lam3, u3, pid);
    PIC_LAUNCHED();
}

template <class Acc>
__global__ void k_acc_to_double(const Acc *a, double *out, int64_t n, double scale) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if constexpr (std::is_same<Acc, double>::value) out[i] = a[i] * scale;
    else out[i] = (double)(long long)a[i] * scale;
}

template <class P>
void launch_acc_to_double(const typename P::Acc *a, double *out, int64_t n, double scale,
                          cudaStream_t s) {
    if (n <= 0) return;
    k_acc_to_double<typename P::Acc><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, out, n, scale);
    PIC_LAUNCHED();
}

#define PIC_INST(P)                                                                            \
    template void launch_diag<P>(const DiagDev &, const P::Acc *, const P::Acc *,              \
                                 const P::Acc *, const P::Acc *, const P::Acc *, const P::Acc *, \
                                 const double *,                                               \
                                 double *, int,                                                \
                                 const P::R *, const P::R *, const P::R *, Particles<P>,       \
                                 const int64_t *, int64_t, double, double, double *,           \
                                 cudaStream_t);                                                \
    template void launch_export<P>(Particles<P>, int64_t, const TriRec<P::R> *, double *,      \
                                   double *, int64_t *, cudaStream_t);                         \
    template void launch_acc_to_double<P>(const P::Acc *, double *, int64_t, double,           \
                                          cudaStream_t);
PIC_INST(PF32)
PIC_INST(PF64)

}  // namespace pic
