// Field probes recorded on the device (the output-port signal of Sec. 5.3 and other
// per-step field reductions), without a host round trip per sample.  After the face
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

}  // namespace

template <class P>
void launch_probe(const ProbeArgs<P> &a, cudaStream_t s) {
    if (a.n_groups <= 0) return;
    k_probe<P><<<(unsigned)a.n_groups, 256, 0, s>>>(a);
    PIC_LAUNCHED();
}

template void launch_probe<PF32>(const ProbeArgs<PF32> &, cudaStream_t);
template void launch_probe<PF64>(const ProbeArgs<PF64> &, cudaStream_t);

}  // namespace pic
