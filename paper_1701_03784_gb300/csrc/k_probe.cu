// Field probes and output-port signals recorded on the device, without a host round trip
// per sample.  After the face
// kernel of a step, group g sums w_k B_f^p_g over its entries (faces f_k, weights w_k,
// power p_g in {1, 2}); every `every` steps the sums of all groups are appended to a
// device buffer.  One block per group; the last block to finish advances the step phase
// and the record count (device counters, so a recorded CUDA graph replays correctly).
#include "pic_internal.h"

namespace pic {

namespace {

template <class P>
__global__ void __launch_bounds__(256) k_probe(ProbeArgs<P> a) {
    __shared__ double part[8];
    __shared__ long long s_step, s_rec;
    __shared__ unsigned ticket;
    if (threadIdx.x == 0) {
        s_step = a.state[0];
        s_rec = a.state[1];
    }
    __syncthreads();
    const bool take = s_step % a.every == 0;
    const int g = blockIdx.x;
    if (take) {
        double s = 0.0;
        const int quad = a.power[g] == 2;
        for (long long k = a.ptr[g] + threadIdx.x; k < a.ptr[g + 1]; k += blockDim.x) {
            const double b = (double)a.B[a.face[k]];
            s += a.weight[k] * (quad ? b * b : b);
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += part[w];
            if (s_rec < a.capacity) a.buf[s_rec * a.n_groups + g] = t;
        }
    }
    // the last block advances the counters
    if (threadIdx.x == 0) {
        __threadfence();
        ticket = atomicAdd(a.done, 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0 && ticket == gridDim.x - 1) {
        a.state[0] = s_step + 1;
        if (take) {
            if (s_rec < a.capacity) a.state[1] = s_rec + 1;
            else a.state[2] += 1;   // records that did not fit
        }
        *a.done = 0;
        __threadfence();
    }
}

// Output-port signal (Secs. 5.1, 5.1.1): the Poynting flux through a plane z = const,
// P = (2 pi / mu0) int E_rho B_phi rho drho, as a quadrature over the triangles the plane
// crosses (the host tabulates points and weights; E_rho and rho are linear along a
// triangle's chord and B_phi constant in it, so two Gauss points per chord are exact).
// E_rho(lambda) = sum_k lambda_k c_k,rho and B_phi come from the triangle records the face
// kernel of this step wrote: E^n and (B^{n+1/2} + B^{n-1/2}) / (2A).  One block per port;
// the step phase and records advance as in k_probe.
template <class P>
__global__ void __launch_bounds__(256) k_port(PortArgs<P> a) {
    __shared__ double part[8];
    __shared__ long long s_step, s_rec;
    __shared__ unsigned ticket;
    if (threadIdx.x == 0) {
        s_step = a.state[0];
        s_rec = a.state[1];
    }
    __syncthreads();
    const bool take = s_step % a.every == 0;
    const int g = blockIdx.x;
    if (take) {
        double s = 0.0;
        for (long long k = a.ptr[g] + threadIdx.x; k < a.ptr[g + 1]; k += blockDim.x) {
            const TriRec<typename P::R> &r = a.rec[a.tri[k]];
            const double *l = a.lam + 3 * k;
            const double er = l[0] * (double)r.c[1] + l[1] * (double)r.c[3] + l[2] * (double)r.c[5];
            s += a.weight[k] * er * (double)r.bphi;
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += part[w];
            if (s_rec < a.capacity) a.buf[s_rec * a.n_ports + g] = t;
        }
    }
    if (threadIdx.x == 0) {
        __threadfence();
        ticket = atomicAdd(a.done, 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0 && ticket == gridDim.x - 1) {
        a.state[0] = s_step + 1;
        if (take) {
            if (s_rec < a.capacity) a.state[1] = s_rec + 1;
            else a.state[2] += 1;
        }
        *a.done = 0;
        __threadfence();
    }
}

}  // namespace

template <class P>
void launch_port(const PortArgs<P> &a, cudaStream_t s) {
    if (a.n_ports <= 0) return;
    k_port<P><<<(unsigned)a.n_ports, 256, 0, s>>>(a);
    PIC_LAUNCHED();
}

template void launch_port<PF32>(const PortArgs<PF32> &, cudaStream_t);
template void launch_port<PF64>(const PortArgs<PF64> &, cudaStream_t);

template <class P>
void launch_probe(const ProbeArgs<P> &a, cudaStream_t s) {
    if (a.n_groups <= 0) return;
    k_probe<P><<<(unsigned)a.n_groups, 256, 0, s>>>(a);
    PIC_LAUNCHED();
}

template void launch_probe<PF32>(const ProbeArgs<PF32> &, cudaStream_t);
template void launch_probe<PF64>(const ProbeArgs<PF64> &, cudaStream_t);

}  // namespace pic
