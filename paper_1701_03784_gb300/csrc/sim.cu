// Simulation object: device-resident fields, operators and particles, and the per-step
// launch sequence of the paper's cycle (Sec. 3).
#include <atomic>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>

#include "pic_internal.h"

namespace pic {

static std::atomic<long long> g_launches{0};
static thread_local long long t_launches = 0;

void note_launches(long long k) {
    g_launches += k;
    t_launches += k;
}
long long launches_this_thread() { return t_launches; }

static Allocator g_allocator;
static std::mutex g_allocator_mu;

Allocator current_allocator() {
    std::lock_guard<std::mutex> lk(g_allocator_mu);
    return g_allocator;
}

// Scratch of pic_charges_get_static: a fixed device array instead of an allocation, for
// callers that must not allocate device memory.  Every GPU that loads the library holds
// these 3 MB until the process exits.  Host code cannot use the symbol itself as a device
// address; the address is looked up once per device (charge_scratch_address).
constexpr int64_t STATIC_MAX_NODES = 131072;
static __device__ __align__(256) double g_charge_scratch[3 * STATIC_MAX_NODES];
static std::mutex g_charge_scratch_mu;
static double *g_charge_scratch_ptr[64] = {nullptr};

// Device address of g_charge_scratch on the current device, resolved on the first call
// per device (cudaGetSymbolAddress, with that device current).
static pic_status charge_scratch_address(double **out) {
    int dev = 0;
    PIC_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        set_error("pic_charges_get_static: device index %d out of range", dev);
        return PIC_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(g_charge_scratch_mu);
    if (!g_charge_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_charge_scratch);
        if (e != cudaSuccess || !p) {
            set_error("pic_charges_get_static: cudaGetSymbolAddress failed: %s",
                      cudaGetErrorString(e));
            return PIC_ERR_CUDA;
        }
        g_charge_scratch_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_charge_scratch_ptr[dev];
    return PIC_OK;
}

struct SimBase {
    virtual ~SimBase() = default;
    virtual pic_status fields_set(const double *E, const double *B, cudaStream_t s) = 0;
    virtual pic_status inject(int64_t n, const double *z, const double *rho, const double *ur,
                              const double *up, const double *uz, double q, double m, double w,
                              cudaStream_t s) = 0;
    virtual pic_status step(int64_t n, cudaStream_t s) = 0;
    virtual pic_status diagnostics(pic_diag *o, double *E, double *B, double *J,
                                   cudaStream_t s) = 0;
    virtual pic_status charges(double *Q, double *Qp, double *Qa, cudaStream_t s) = 0;
    virtual pic_status count(int64_t *n, cudaStream_t s) = 0;
    virtual pic_status get(int64_t cap, int64_t *pid, int32_t *tri, double *lam, double *u,
                           cudaStream_t s) = 0;
    virtual int64_t raw_bytes() const = 0;
    // slots per array in the raw host layout: n rounded up to 32, so that every array
    // starts on a 128-byte boundary (host -> device copies from a less aligned start ran
    // at 177 instead of 210 GB/s)
    static int64_t raw_stride(int64_t n) { return (n + 31) / 32 * 32; }
    virtual pic_status raw_get(void *dst, int64_t n, cudaStream_t s) = 0;
    virtual pic_status raw_set(const void *src, int64_t n, cudaStream_t s) = 0;
    virtual pic_status step_host(void *state, int64_t n, int64_t steps, cudaStream_t s) = 0;
    virtual void set_graph(bool on) = 0;
    virtual pic_status autotune(int32_t trial, pic_tuning *out, cudaStream_t s) = 0;
    virtual pic_status timing(int enable, double *ms, int64_t *launches, cudaStream_t s) = 0;
    virtual pic_status charges_static(double *Q, double *Qp, double *Qa, cudaStream_t s) = 0;
    virtual pic_status set_static_field(const double *E, cudaStream_t s) = 0;
    virtual pic_status set_emitter(const pic_emitter *e, cudaStream_t s) = 0;
    virtual pic_status set_loss(const double *sig_e, const double *sig_m, cudaStream_t s) = 0;
    virtual pic_status set_probes(int64_t n, const int32_t *face, const int32_t *group,
                                  const double *weight, int32_t n_groups, const int32_t *power,
                                  int64_t capacity, int32_t every, cudaStream_t s) = 0;
    virtual pic_status probes_read(double *out, int64_t cap, int64_t *n_rec, int64_t *n_drop,
                                   cudaStream_t s) = 0;
    virtual pic_status set_ports(int32_t n, const double *z, const double *rho0,
                                 const double *rho1, int64_t capacity, int32_t every,
                                 cudaStream_t s) = 0;
    virtual pic_status ports_read(double *out, int64_t cap, int64_t *n_rec, int64_t *n_drop,
                                  cudaStream_t s) = 0;
    int32_t sort_interval = 16;
    int32_t pusher = PIC_PUSHER_BORIS;
    int64_t wait_polls = PUSH_WAIT_POLLS;   // particle kernel's tile-pipeline waits
    int device = 0;
};

// live slots of each of nch ranges of `chunk` slots, from the device slot count *n (which a
// re-sort may have lowered below the host's count)
__global__ void k_chunk_counts(const int64_t *n, int64_t *out, int64_t chunk, int nch) {
    const int c = threadIdx.x;
    if (c < nch) {
        const int64_t r = *n - (int64_t)c * chunk;
        out[c] = r < 0 ? 0 : (r > chunk ? chunk : r);
    }
}

template <class P>
struct SimImpl final : SimBase {
    using R = typename P::R;
    using Acc = typename P::Acc;
    using Lam = typename P::Lam;

    const HostMesh *m = nullptr;
    Allocator al;
    std::vector<void *> allocs;
    double dt = 0, bz = 0, q = 0, mass = 0, weight = 0, q_src = 0, qm = 0;
    bool have_species = false;
    int64_t cap = 0, n_bound = 0, next_pid = 0, n_steps = 0, n_injected = 0;
    int cur = 0, qcur = 0, since_sort = 0;
    bool dgl_dirty = true;
    int64_t nf = 0, n_slices = 0;

    TriRec<R> *rec = nullptr;
    R *E = nullptr, *B = nullptr, *mu_inv = nullptr, *r = nullptr;
    int32_t *edge_face = nullptr, *free_edges = nullptr;
    double *D = nullptr;
    int64_t *ell_off = nullptr;
    int32_t *ell_col = nullptr;
    R *ell_val = nullptr;
    Acc *J = nullptr, *Qbuf[2] = {nullptr, nullptr}, *Qabs = nullptr, *qpos = nullptr;
    Acc *Qwall = nullptr;   // charge removed at walls since the Gauss-law reference
    Particles<P> parts[2];
    int64_t *d_n = nullptr;
    unsigned long long *counters = nullptr;
    SortScratch sc;
    DiagDev dd{};
    double *dgl_ref = nullptr, *diag_out = nullptr;
    // sources (Secs. 5.2, 5.3): a static field added at the gather, and an emitter
    R *Es = nullptr;
    bool static_on = false, emitting = false, emitter_ever = false;
    pic_emitter em{};
    EmitLine eline{};
    double *el_buf = nullptr;
    int32_t *el_tri = nullptr;
    int64_t el_room = 0;
    int src_version = 0;
    // lossy layer: per free edge and per face (a, b) update factors, and the Gauss-law
    // node mask with the layer's nodes added (conduction moves charge there)
    R *loss_e = nullptr, *loss_f = nullptr;
    bool loss_on = false;
    const uint8_t *pec_mask = nullptr;
    uint8_t *dgl_mask = nullptr;
    // field probes recorded on the device
    ProbeArgs<P> probe{};
    bool probes_on = false;
    // output ports recorded on the device
    PortArgs<P> port{};
    bool ports_on = false;

    bool timing_on = false;
    // host round trips (step_host): uploads and downloads run on streams of their own,
    // chunk by chunk (16M slots, ms per step: 2, 3, 4, 6, 8, 16, 32 chunks -> 2.63, 2.53,
    // 2.57, 2.66, 2.75, 3.15, 3.15; each chunk costs a particle-kernel launch and six
    // copies each way, more than the shorter pipeline tail saves)
    static constexpr int RT_CHUNKS = 3;
    // CUDA-graph replay of whole periods of steps (2 x the re-sort interval: the buffer
    // parities and the re-sort phase are back where they started)
    bool use_graph = false, stepped = false;
    // launch shapes chosen by autotune: persistent CTAs per SM of the particle kernel
    // (0: as many as fit) and threads per block of the field kernels
    int32_t tune_ctas = 0, tune_block = 256;
    cudaStream_t g_stream = nullptr;
    cudaGraphExec_t g_exec = nullptr;
    int g_cur = 0, g_qcur = 0, g_since = 0, g_interval = -1, g_ctas = -1, g_block = -1, g_pusher = -1,
        g_src = -1;
    int64_t g_bound = -1, g_wait = -1;
    long long g_kernels = 0;   // kernels recorded in g_exec
    cudaStream_t rt_stream = nullptr, up_stream = nullptr;
    cudaEvent_t rt_chunk[RT_CHUNKS] = {}, rt_step = nullptr, rt_done = nullptr, rt_up = nullptr;
    cudaEvent_t rt_upc[RT_CHUNKS] = {}, rt_pushc[RT_CHUNKS] = {};   // a chunk uploaded / pushed
    int64_t *d_chunk_n = nullptr;                                    // live slots per chunk
    std::vector<cudaEvent_t> ev_free;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending;

    ~SimImpl() override {
        cudaSetDevice(device);
        cudaDeviceSynchronize();
        if (g_exec) cudaGraphExecDestroy(g_exec);
        if (g_stream) cudaStreamDestroy(g_stream);
        if (rt_stream) {
            for (auto e : rt_chunk) cudaEventDestroy(e);
            for (auto e : rt_upc) cudaEventDestroy(e);
            for (auto e : rt_pushc) cudaEventDestroy(e);
            cudaEventDestroy(rt_step);
            cudaEventDestroy(rt_done);
            cudaEventDestroy(rt_up);
            cudaStreamDestroy(rt_stream);
            cudaStreamDestroy(up_stream);
        }
        for (auto &e : ev_pending) {
            cudaEventDestroy(e.first);
            cudaEventDestroy(e.second);
        }
        for (auto e : ev_free) cudaEventDestroy(e);
        for (void *p : allocs) {
            if (al.free) al.free(p, al.ctx);
            else cudaFree(p);
        }
    }

    template <class T>
    pic_status dalloc(T *&p, int64_t n) {
        size_t bytes = sizeof(T) * (size_t)std::max<int64_t>(n, 1);
        void *v = nullptr;
        if (al.alloc) {
            v = al.alloc(bytes, al.ctx);
            if (!v) {
                set_error("device allocation of %zu bytes failed", bytes);
                return PIC_ERR_OOM;
            }
        } else {
            cudaError_t e = cudaMalloc(&v, bytes);
            if (e != cudaSuccess) {
                set_error("cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
                return e == cudaErrorMemoryAllocation ? PIC_ERR_OOM : PIC_ERR_CUDA;
            }
        }
        allocs.push_back(v);
        p = static_cast<T *>(v);
        return PIC_OK;
    }

    template <class T>
    pic_status upload(T *&p, const std::vector<T> &h) {
        pic_status st = dalloc(p, (int64_t)h.size());
        if (st != PIC_OK) return st;
        if (!h.empty()) PIC_CUDA_TRY(cudaMemcpy(p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
        return PIC_OK;
    }

    pic_status init(const HostMesh &mesh, double dt_, double bz_, int64_t cap_) {
        m = &mesh;
        dt = dt_;
        bz = bz_;
        cap = cap_;
        nf = (int64_t)mesh.free_edges.size();
        PIC_CUDA_TRY(cudaGetDevice(&device));
        pic_status st;
        // triangle records
        std::vector<TriRec<R>> hr(mesh.N2);
        for (int64_t t = 0; t < mesh.N2; t++) {
            TriRec<R> &x = hr[t];
            std::memset(&x, 0, sizeof x);
            for (int k = 0; k < 4; k++) x.g[k] = (R)mesh.grad[6 * t + k];
            int flags = 0;
            for (int k = 0; k < 3; k++) {
                int32_t nk = mesh.tri[3 * t + k];
                x.node[k] = nk;
                x.rho[k] = (R)mesh.zr[2 * nk + 1];
                x.edge[k] = mesh.tri_edge[3 * t + k];
                int32_t nb = mesh.tri_nbr[3 * t + k];
                x.nbr[k] = nb >= 0 ? nb : -mesh.edge_tag[mesh.tri_edge[3 * t + k]];
                if (mesh.tri[3 * t + (k + 1) % 3] < mesh.tri[3 * t + (k + 2) % 3]) flags |= 1 << k;
            }
            x.flags = flags;
            x.eflags = flags;
            int entry = 0;
            for (int k = 0; k < 3; k++) {
                const int32_t nb = mesh.tri_nbr[3 * t + k];
                if (nb < 0) continue;
                const int32_t ga = mesh.tri[3 * t + (k + 1) % 3], gb = mesh.tri[3 * t + (k + 2) % 3];
                for (int j = 0; j < 3; j++) {
                    const int32_t q = mesh.tri[3 * nb + j];
                    if (q != ga && q != gb) entry |= j << (2 * k);
                }
            }
            x.entry = entry;
            x.inv_area = (R)(1.0 / mesh.area[t]);
        }
        if ((st = upload(rec, hr)) != PIC_OK) return st;
        std::vector<R> hmu(mesh.mu_inv.begin(), mesh.mu_inv.end());
        if ((st = upload(mu_inv, hmu)) != PIC_OK) return st;
        // the two faces of each free edge, in free-edge order
        std::vector<int32_t> hef(2 * std::max<int64_t>(nf, 1), 0);
        for (int64_t i = 0; i < nf; i++) {
            const int64_t e = mesh.free_edges[i];
            for (int q2 = 0; q2 < 2; q2++) {
                int32_t f = mesh.edge_face[2 * e + q2];
                if (f >= 0) hef[2 * i + q2] = (f + 1) * mesh.edge_face_sign[2 * e + q2];
            }
        }
        if ((st = upload(edge_face, hef)) != PIC_OK) return st;
        if ((st = upload(free_edges, mesh.free_edges)) != PIC_OK) return st;
        // M as sliced ELL (slices of 32 rows, column-major inside a slice)
        n_slices = (nf + 31) / 32;
        std::vector<int64_t> hoff(n_slices + 1, 0);
        for (int64_t sl = 0; sl < n_slices; sl++) {
            int64_t w = 0;
            for (int64_t i = sl * 32; i < std::min(nf, sl * 32 + 32); i++)
                w = std::max<int64_t>(w, mesh.M_ptr[i + 1] - mesh.M_ptr[i]);
            hoff[sl + 1] = hoff[sl] + 32 * w;
        }
        std::vector<int32_t> hcol(std::max<int64_t>(hoff[n_slices], 1), 0);
        std::vector<R> hval(std::max<int64_t>(hoff[n_slices], 1), R(0));
        for (int64_t i = 0; i < nf; i++) {
            int64_t sl = i / 32, lane = i % 32, k = 0;
            for (int64_t q2 = mesh.M_ptr[i]; q2 < mesh.M_ptr[i + 1]; q2++, k++) {
                hcol[hoff[sl] + 32 * k + lane] = mesh.M_idx[q2];
                hval[hoff[sl] + 32 * k + lane] = (R)mesh.M_val[q2];
            }
        }
        if ((st = upload(ell_off, hoff)) != PIC_OK) return st;
        if ((st = upload(ell_col, hcol)) != PIC_OK) return st;
        if ((st = upload(ell_val, hval)) != PIC_OK) return st;
        // fields and accumulators
        if ((st = dalloc(E, mesh.N1)) || (st = dalloc(B, mesh.N2)) || (st = dalloc(D, mesh.N1)) ||
            (st = dalloc(r, nf)) || (st = dalloc(J, mesh.N1)) || (st = dalloc(Qbuf[0], mesh.N0)) ||
            (st = dalloc(Qbuf[1], mesh.N0)) || (st = dalloc(Qabs, mesh.N0)) || (st = dalloc(Qwall, mesh.N0)) ||
            (st = dalloc(qpos, mesh.N0)))
            return st;
        PIC_CUDA_TRY(cudaMemset(E, 0, sizeof(R) * mesh.N1));
        PIC_CUDA_TRY(cudaMemset(B, 0, sizeof(R) * mesh.N2));
        PIC_CUDA_TRY(cudaMemset(D, 0, sizeof(double) * mesh.N1));
        PIC_CUDA_TRY(cudaMemset(J, 0, sizeof(Acc) * mesh.N1));
        for (int k = 0; k < 2; k++) PIC_CUDA_TRY(cudaMemset(Qbuf[k], 0, sizeof(Acc) * mesh.N0));
        PIC_CUDA_TRY(cudaMemset(Qabs, 0, sizeof(Acc) * mesh.N0));
        // particles, double-buffered for the re-sort
        for (int k = 0; k < 2; k++) {
            Particles<P> &p = parts[k];
            const int64_t ca = cap + SLOT_PAD;  // bulk copies round up to 16 bytes
            if ((st = dalloc(p.tri, ca)) || (st = dalloc(p.l0, ca)) || (st = dalloc(p.l1, ca)) ||
                (st = dalloc(p.ur, ca)) || (st = dalloc(p.up, ca)) || (st = dalloc(p.uz, ca)) ||
                (st = dalloc(p.pid, ca)))
                return st;
        }
        if ((st = dalloc(d_n, 1)) || (st = dalloc(counters, CNT_N))) return st;
        PIC_CUDA_TRY(cudaMemset(d_n, 0, sizeof(int64_t)));
        PIC_CUDA_TRY(cudaMemset(counters, 0, sizeof(unsigned long long) * CNT_N));
        // sort scratch
        if ((st = dalloc(sc.cnt, mesh.N2 + 1)) || (st = dalloc(sc.blk, mesh.N2 / 2048 + 2)) ||
            (st = dalloc(sc.n_old, 1)))
            return st;
        // diagnostics: node -> edge incidence (D_div rows), star_eps
        std::vector<int64_t> nptr(mesh.N0 + 1, 0);
        for (int64_t e = 0; e < mesh.N1; e++) {
            nptr[mesh.edge_nodes[2 * e] + 1]++;
            nptr[mesh.edge_nodes[2 * e + 1] + 1]++;
        }
        for (int64_t k = 0; k < mesh.N0; k++) nptr[k + 1] += nptr[k];
        std::vector<int32_t> nedge(nptr[mesh.N0]);
        std::vector<int8_t> nsign(nptr[mesh.N0]);
        std::vector<int64_t> fill(nptr.begin(), nptr.end() - 1);
        for (int64_t e = 0; e < mesh.N1; e++) {
            int32_t a = mesh.edge_nodes[2 * e], b = mesh.edge_nodes[2 * e + 1];
            nedge[fill[a]] = (int32_t)e;
            nsign[fill[a]++] = 1;   // current leaves the tail
            nedge[fill[b]] = (int32_t)e;
            nsign[fill[b]++] = -1;
        }
        int64_t *np_ = nullptr, *ep_ = nullptr;
        int32_t *ne_ = nullptr, *ei_ = nullptr;
        int8_t *ns_ = nullptr;
        uint8_t *pec_ = nullptr;
        double *ev_ = nullptr;
        std::vector<int64_t> eptr(mesh.eps_ptr.begin(), mesh.eps_ptr.end());
        if ((st = upload(np_, nptr)) || (st = upload(ne_, nedge)) || (st = upload(ns_, nsign)) ||
            (st = upload(pec_, mesh.node_on_pec)) || (st = upload(ep_, eptr)) ||
            (st = upload(ei_, mesh.eps_idx)) || (st = upload(ev_, mesh.eps_val)))
            return st;
        dd = DiagDev{np_, ne_, ns_, pec_, ep_, ei_, ev_, mesh.N0, mesh.N1, mesh.N2};
        pec_mask = pec_;
        if ((st = dalloc(dgl_ref, mesh.N0)) || (st = dalloc(diag_out, 8))) return st;
        PIC_CUDA_TRY(cudaDeviceSynchronize());
        return PIC_OK;
    }

    Acc *Qn() { return Qbuf[qcur]; }
    double j_scale() const { return (P::fixed ? J_INV : 1.0) * q_src / dt; }
    double q_scale() const { return q_src; }

    FieldArgs<P> field_args() {
        FieldArgs<P> a;
        a.rec = rec;
        a.E = E;
        a.B = B;
        a.mu_inv = mu_inv;
        a.edge_face = edge_face;
        a.free_edges = free_edges;
        a.J = J;
        a.D = D;
        a.r = r;
        a.ell_off = ell_off;
        a.ell_col = ell_col;
        a.ell_val = ell_val;
        a.N1 = m->N1;
        a.N2 = m->N2;
        a.nf = nf;
        a.dt = (R)dt;
        a.j_scale = j_scale();
        a.node_ptr = dd.node_ptr;
        a.node_edge = dd.node_edge;
        a.node_sign = dd.node_sign;
        a.Qn = nullptr;
        a.Qabs = Qabs;
        a.Qnext = nullptr;
        a.Qwall = Qwall;
        a.counters = counters;
        a.N0 = m->N0;
        a.block = tune_block;
        a.Es = static_on ? Es : nullptr;
        a.loss_e = loss_on ? loss_e : nullptr;
        a.loss_f = loss_on ? loss_f : nullptr;
        return a;
    }

    pic_status set_probes(int64_t n, const int32_t *face, const int32_t *group, const double *weight,
                          int32_t n_groups, const int32_t *power, int64_t capacity, int32_t every,
                          cudaStream_t s) override {
        src_version++;
        if (n <= 0 || n_groups <= 0) {
            probes_on = false;
            return PIC_OK;
        }
        if (!face || !group || !weight || !power || capacity < 1 || every < 1) {
            set_error("pic_sim_set_probes: bad argument");
            return PIC_ERR_ARG;
        }
        std::vector<int64_t> ptr(n_groups + 1, 0);
        for (int64_t k = 0; k < n; k++) {
            if (face[k] < 0 || face[k] >= m->N2 || group[k] < 0 || group[k] >= n_groups ||
                !std::isfinite(weight[k])) {
                set_error("pic_sim_set_probes: entry %lld out of range", (long long)k);
                return PIC_ERR_ARG;
            }
            ptr[group[k] + 1]++;
        }
        for (int32_t g = 0; g < n_groups; g++) {
            if (power[g] != 1 && power[g] != 2) {
                set_error("pic_sim_set_probes: power of group %d is not 1 or 2", (int)g);
                return PIC_ERR_ARG;
            }
            ptr[g + 1] += ptr[g];
        }
        std::vector<int32_t> f(n);
        std::vector<double> w(n);
        std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
        for (int64_t k = 0; k < n; k++) {
            const int64_t at = fill[group[k]]++;
            f[at] = face[k];
            w[at] = weight[k];
        }
        std::vector<int32_t> pw(power, power + n_groups);
        int64_t *d_ptr;
        int32_t *d_face, *d_pow;
        double *d_w, *d_buf;
        long long *d_state;
        unsigned *d_done;
        pic_status st;
        if ((st = upload(d_ptr, ptr)) || (st = upload(d_face, f)) || (st = upload(d_w, w)) ||
            (st = upload(d_pow, pw)) || (st = dalloc(d_buf, capacity * (int64_t)n_groups)) ||
            (st = dalloc(d_state, 3)) || (st = dalloc(d_done, 1)))
            return st;
        PIC_CUDA_TRY(cudaMemsetAsync(d_state, 0, 3 * sizeof(long long), s));
        PIC_CUDA_TRY(cudaMemsetAsync(d_done, 0, sizeof(unsigned), s));
        PIC_CUDA_TRY(cudaStreamSynchronize(s));
        probe = ProbeArgs<P>{B, d_ptr, d_face, d_w, d_pow, d_buf, d_state, d_done, n_groups, every,
                             (long long)capacity};
        probes_on = true;
        return PIC_OK;
    }

    pic_status probes_read(double *out, int64_t cap_rec, int64_t *n_rec, int64_t *n_drop,
                           cudaStream_t s) override {
        if (!probes_on) {
            set_error("pic_probes_read: no probes set");
            return PIC_ERR_STATE;
        }
        long long st3[3];
        PIC_CUDA_TRY(cudaMemcpyAsync(st3, probe.state, sizeof st3, cudaMemcpyDeviceToHost, s));
        PIC_CUDA_TRY(cudaStreamSynchronize(s));
        const int64_t rec = std::min<int64_t>(st3[1], cap_rec);
        if (out && rec > 0)
            PIC_CUDA_TRY(cudaMemcpyAsync(out, probe.buf, sizeof(double) * rec * probe.n_groups,
                                         cudaMemcpyDeviceToHost, s));
        // the records are consumed; the step phase carries on
        PIC_CUDA_TRY(cudaMemsetAsync(probe.state + 1, 0, 2 * sizeof(long long), s));
        PIC_CUDA_TRY(cudaStreamSynchronize(s));
        if (n_rec) *n_rec = rec;
        if (n_drop) *n_drop = st3[2] + (st3[1] - rec);
        return PIC_OK;
    }

    // Output ports: for each plane z_k, the chords of the triangles it crosses between
    // rho0_k and rho1_k (the emission line's tabulation), two Gauss-Legendre points per
    // chord with weights (2 pi / mu0) (rho_b - rho_a) / 2 rho.
    pic_status set_ports(int32_t n, const double *z, const double *rho0, const double *rho1,
                         int64_t capacity, int32_t every, cudaStream_t s) override {
        src_version++;
        if (n <= 0) {
            ports_on = false;
            return PIC_OK;
        }
        if (!z || !rho0 || !rho1 || capacity < 1 || every < 1) {
            set_error("pic_sim_set_ports: bad argument");
            return PIC_ERR_ARG;
        }
        const double gp = 0.5 / std::sqrt(3.0);
        const double pi2_mu = 2.0 * M_PI / m->units.mu0;
        std::vector<int64_t> ptr(n + 1, 0);
        std::vector<int32_t> tri;
        std::vector<double> lam, w;
        for (int32_t k = 0; k < n; k++) {
            std::vector<double> ra, rb, la, lb;
            std::vector<int32_t> tr;
            if (!std::isfinite(z[k]) || !(rho1[k] > rho0[k]) || rho0[k] < 0.0 ||
                !build_emit_line(*m, z[k], rho0[k], rho1[k], ra, rb, la, lb, tr)) {
                set_error("pic_sim_set_ports: port %d (z = %g, rho in [%g, %g]) does not cross "
                          "the mesh in one piece", (int)k, z[k], rho0[k], rho1[k]);
                return PIC_ERR_ARG;
            }
            for (size_t i = 0; i < tr.size(); i++) {
                for (int g = 0; g < 2; g++) {
                    const double f = g == 0 ? 0.5 - gp : 0.5 + gp;
                    const double rho = ra[i] + f * (rb[i] - ra[i]);
                    tri.push_back(tr[i]);
                    for (int c = 0; c < 3; c++)
                        lam.push_back(la[3 * i + c] + f * (lb[3 * i + c] - la[3 * i + c]));
                    w.push_back(pi2_mu * 0.5 * (rb[i] - ra[i]) * rho);
                }
            }
            ptr[k + 1] = (int64_t)tri.size();
        }
        int64_t *d_ptr;
        int32_t *d_tri;
        double *d_lam, *d_w, *d_buf;
        long long *d_state;
        unsigned *d_done;
        pic_status st;
        if ((st = upload(d_ptr, ptr)) || (st = upload(d_tri, tri)) || (st = upload(d_lam, lam)) ||
            (st = upload(d_w, w)) || (st = dalloc(d_buf, capacity * (int64_t)n)) ||
            (st = dalloc(d_state, 3)) || (st = dalloc(d_done, 1)))
            return st;
        PIC_CUDA_TRY(cudaMemsetAsync(d_state, 0, 3 * sizeof(long long), s));
        PIC_CUDA_TRY(cudaMemsetAsync(d_done, 0, sizeof(unsigned), s));
        PIC_CUDA_TRY(cudaStreamSynchronize(s));
        port = PortArgs<P>{rec, d_ptr, d_tri, d_lam, d_w, d_buf, d_state, d_done, n, every,
                           (long long)capacity};
        ports_on = true;
        return PIC_OK;
    }

    pic_status ports_read(double *out, int64_t cap_rec, int64_t *n_rec, int64_t *n_drop,
                          cudaStream_t s) override {
        if (!ports_on) {
            set_error("pic_ports_read: no ports set");
            return PIC_ERR_STATE;
        }
        long long st3[3];
        PIC_CUDA_TRY(cudaMemcpyAsync(st3, port.state, sizeof st3, cudaMemcpyDeviceToHost, s));
        PIC_CUDA_TRY(cudaStreamSynchronize(s));
        const int64_t rec_n = std::min<int64_t>(st3[1], cap_rec);
        if (out && rec_n > 0)
            PIC_CUDA_TRY(cudaMemcpyAsync(out, port.buf, sizeof(double) * rec_n * port.n_ports,
                                         cudaMemcpyDeviceToHost, s));
        PIC_CUDA_TRY(cudaMemsetAsync(port.state + 1, 0, 2 * sizeof(long long), s));
        PIC_CUDA_TRY(cudaStreamSynchronize(s));
        if (n_rec) *n_rec = rec_n;
        if (n_drop) *n_drop = st3[2] + (st3[1] - rec_n);
        return PIC_OK;
    }

    pic_status set_loss(const double *sig_e, const double *sig_m, cudaStream_t s) override {
        src_version++;
        if (!sig_e && !sig_m) {
            loss_on = false;
            dd.node_on_pec = pec_mask;
            dgl_dirty = true;
            return PIC_OK;
        }
        const double eps0 = m->units.eps0, mu0 = m->units.mu0;
        std::vector<R> le(2 * nf), lf(2 * m->N2);
        std::vector<uint8_t> mask(m->node_on_pec.begin(), m->node_on_pec.end());
        for (int64_t i = 0; i < nf; i++) {
            const int32_t e = m->free_edges[i];
            const double sg = sig_e ? sig_e[e] : 0.0;
            if (!(sg >= 0.0) || !std::isfinite(sg)) {
                set_error("pic_sim_set_loss: edge conductivity %lld negative or not finite", (long long)e);
                return PIC_ERR_ARG;
            }
            const double x = sg * dt / (2.0 * eps0);
            le[2 * i] = (R)((1.0 - x) / (1.0 + x));
            le[2 * i + 1] = (R)(1.0 / (1.0 + x));
            if (sg > 0.0) mask[m->edge_nodes[2 * e]] = mask[m->edge_nodes[2 * e + 1]] = 1;
        }
        for (int64_t f = 0; f < m->N2; f++) {
            const double sg = sig_m ? sig_m[f] : 0.0;
            if (!(sg >= 0.0) || !std::isfinite(sg)) {
                set_error("pic_sim_set_loss: face conductivity %lld negative or not finite", (long long)f);
                return PIC_ERR_ARG;
            }
            const double x = sg * dt / (2.0 * mu0);
            lf[2 * f] = (R)((1.0 - x) / (1.0 + x));
            lf[2 * f + 1] = (R)(1.0 / (1.0 + x));
            if (sg > 0.0)
                for (int k = 0; k < 3; k++) mask[m->tri[3 * f + k]] = 1;
        }
        pic_status st;
        if (!loss_e && ((st = dalloc(loss_e, 2 * nf)) != PIC_OK || (st = dalloc(loss_f, 2 * m->N2)) != PIC_OK ||
                        (st = dalloc(dgl_mask, m->N0)) != PIC_OK))
            return st;
        PIC_CUDA_TRY(cudaMemcpyAsync(loss_e, le.data(), sizeof(R) * 2 * nf, cudaMemcpyHostToDevice, s));
        PIC_CUDA_TRY(cudaMemcpyAsync(loss_f, lf.data(), sizeof(R) * 2 * m->N2, cudaMemcpyHostToDevice, s));
        PIC_CUDA_TRY(cudaMemcpyAsync(dgl_mask, mask.data(), m->N0, cudaMemcpyHostToDevice, s));
        PIC_CUDA_TRY(cudaStreamSynchronize(s));
        dd.node_on_pec = dgl_mask;
        loss_on = true;
        dgl_dirty = true;   // the reference is taken again over the new node set
        return PIC_OK;
    }

    pic_status set_static_field(const double *Eh, cudaStream_t s) override {
        src_version++;
        if (!Eh) {
            static_on = false;
            return PIC_OK;
        }
        std::vector<R> e(m->N1);
        for (int64_t i = 0; i < m->N1; i++) {
            if (!std::isfinite(Eh[i])) {
                set_error("pic_sim_set_static_field: edge value %lld is not finite", (long long)i);
                return PIC_ERR_ARG;
            }
            e[i] = (R)Eh[i];
        }
        pic_status st;
        if (!Es && (st = dalloc(Es, m->N1)) != PIC_OK) return st;
        PIC_CUDA_TRY(cudaMemcpyAsync(Es, e.data(), sizeof(R) * m->N1, cudaMemcpyHostToDevice, s));
        PIC_CUDA_TRY(cudaStreamSynchronize(s));
        static_on = true;
        return PIC_OK;
    }

    pic_status set_emitter(const pic_emitter *e, cudaStream_t s) override {
        src_version++;
        if (!e) {
            emitting = false;
            return PIC_OK;
        }
        if (e->per_step < 0 || !(e->rho0 >= 0.0) || !(e->rho1 > e->rho0) || !std::isfinite(e->z) ||
            !std::isfinite(e->u_normal) || !(e->u_thermal >= 0.0) || !(e->m > 0) || !(e->w > 0) ||
            !std::isfinite(e->q)) {
            set_error("pic_sim_set_emitter: bad argument");
            return PIC_ERR_ARG;
        }
        const double qsrc = e->w * e->q / (2.0 * M_PI);
        if (have_species && (e->q / e->m != qm || qsrc != q_src)) {
            set_error("pic_sim_set_emitter: one species per simulation (q/m and q*w must match)");
            return PIC_ERR_ARG;
        }
        std::vector<double> ra, rb, la, lb;
        std::vector<int32_t> tr;
        if (!build_emit_line(*m, e->z, e->rho0, e->rho1, ra, rb, la, lb, tr)) {
            set_error("pic_sim_set_emitter: the line z = %g, rho in [%g, %g] does not lie inside "
                      "the mesh, or meets a node", e->z, e->rho0, e->rho1);
            return PIC_ERR_ARG;
        }
        const int64_t n = (int64_t)tr.size();
        pic_status st;
        if (n > el_room) {
            if ((st = dalloc(el_buf, 8 * n)) != PIC_OK || (st = dalloc(el_tri, n)) != PIC_OK) return st;
            el_room = n;
        }
        std::vector<double> buf(8 * n);
        std::copy(ra.begin(), ra.end(), buf.begin());
        std::copy(rb.begin(), rb.end(), buf.begin() + n);
        std::copy(la.begin(), la.end(), buf.begin() + 2 * n);
        std::copy(lb.begin(), lb.end(), buf.begin() + 5 * n);
        PIC_CUDA_TRY(cudaMemcpyAsync(el_buf, buf.data(), sizeof(double) * 8 * n, cudaMemcpyHostToDevice, s));
        PIC_CUDA_TRY(cudaMemcpyAsync(el_tri, tr.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
        if (!emitter_ever) {
            // particle ids continue on the device from here on
            unsigned long long np = (unsigned long long)next_pid;
            PIC_CUDA_TRY(cudaMemcpyAsync(counters + CNT_NEXT_PID, &np, sizeof np, cudaMemcpyHostToDevice, s));
        }
        PIC_CUDA_TRY(cudaStreamSynchronize(s));
        eline = EmitLine{el_buf, el_buf + n, el_buf + 2 * n, el_buf + 5 * n, el_tri, (int32_t)n};
        em = *e;
        if (!have_species) {
            have_species = true;
            q = e->q;
            mass = e->m;
            weight = e->w;
            qm = e->q / e->m;
            q_src = qsrc;
        }
        emitting = true;
        emitter_ever = true;
        // launches cover the whole capacity from now on (the kernels read the live count)
        n_bound = cap;
        return PIC_OK;
    }

    pic_status fields_set(const double *Eh, const double *Bh, cudaStream_t s) override {
        if (Eh) {
            std::vector<R> e(m->N1);
            std::vector<double> ed(m->N1);
            for (int64_t i = 0; i < m->N1; i++) {
                double v = m->edge_tag[i] == PIC_BC_PEC ? 0.0 : Eh[i];
                ed[i] = v;
                e[i] = (R)v;
            }
            // auxiliary dual flux D = star_eps E (Sec. 3.5.2)
            std::vector<double> dh(m->N1, 0.0);
            for (int64_t i = 0; i < m->N1; i++) {
                double acc = 0;
                for (int64_t k = m->eps_ptr[i]; k < m->eps_ptr[i + 1]; k++)
                    acc += m->eps_val[k] * (double)e[m->eps_idx[k]];
                dh[i] = acc;
            }
            PIC_CUDA_TRY(cudaMemcpyAsync(E, e.data(), sizeof(R) * m->N1, cudaMemcpyHostToDevice, s));
            PIC_CUDA_TRY(cudaMemcpyAsync(D, dh.data(), sizeof(double) * m->N1, cudaMemcpyHostToDevice, s));
            PIC_CUDA_TRY(cudaStreamSynchronize(s));
        }
        if (Bh) {
            std::vector<R> b(Bh, Bh + m->N2);
            PIC_CUDA_TRY(cudaMemcpyAsync(B, b.data(), sizeof(R) * m->N2, cudaMemcpyHostToDevice, s));
            PIC_CUDA_TRY(cudaStreamSynchronize(s));
        }
        dgl_dirty = true;
        return PIC_OK;
    }

    pic_status read_count(int64_t *n, cudaStream_t s) {
        PIC_CUDA_TRY(cudaMemcpyAsync(n, d_n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        PIC_CUDA_TRY(cudaStreamSynchronize(s));
        return PIC_OK;
    }

    pic_status resort(cudaStream_t s) {
        launch_resort<P>(parts[cur], parts[1 - cur], d_n, n_bound, m->N2, sc, s);
        cur = 1 - cur;
        since_sort = 0;
        return PIC_OK;
    }

    pic_status inject(int64_t n, const double *z, const double *rho, const double *ur,
                      const double *up, const double *uz, double q_, double m_, double w_,
                      cudaStream_t s) override {
        if (n < 0 || (n > 0 && (!z || !rho || !ur || !up || !uz)) || !(m_ > 0) || !(w_ > 0) ||
            !std::isfinite(q_)) {
            set_error("pic_particles_inject: bad argument");
            return PIC_ERR_ARG;
        }
        double qsrc = w_ * q_ / (2.0 * M_PI);
        if (have_species && (q_ / m_ != qm || qsrc != q_src)) {
            set_error("pic_particles_inject: one species per simulation (q/m and q*w must match)");
            return PIC_ERR_ARG;
        }
        if (n == 0) return PIC_OK;
        int64_t n_now = 0;
        pic_status st = read_count(&n_now, s);
        if (st != PIC_OK) return st;
        if (n_now + n > cap) {
            set_error("pic_particles_inject: capacity %lld exceeded", (long long)cap);
            return PIC_ERR_OOM;
        }
        if (emitter_ever) {
            // the emitter numbers particles on the device: continue from its count
            unsigned long long np = 0;
            PIC_CUDA_TRY(cudaMemcpyAsync(&np, counters + CNT_NEXT_PID, sizeof np, cudaMemcpyDeviceToHost, s));
            PIC_CUDA_TRY(cudaStreamSynchronize(s));
            next_pid = (int64_t)np;
        }
        std::vector<int32_t> tri(n), pid(n);
        std::vector<Lam> l0(n), l1(n);
        std::vector<R> vr(n), vp(n), vz(n);
        std::vector<uint8_t> bad(1, 0);
        const HostMesh &mm = *m;
        parallel_for(n, [&](int64_t a, int64_t b) {
            for (int64_t i = a; i < b; i++) {
                double lam[3];
                int32_t t = locate_point(mm, z[i], rho[i], lam);
                if (t < 0 || !std::isfinite(ur[i] + up[i] + uz[i])) {
                    bad[0] = 1;
                    continue;
                }
                tri[i] = t;
                if constexpr (P::fixed) {
                    // integers that sum to 2^22
                    double a0 = std::max(lam[0], 0.0), a1 = std::max(lam[1], 0.0),
                           a2 = std::max(lam[2], 0.0);
                    double ss = a0 + a1 + a2;
                    int32_t q0 = (int32_t)std::nearbyint(a0 / ss * LAM_ONE);
                    int32_t q1 = (int32_t)std::nearbyint(a1 / ss * LAM_ONE);
                    int32_t q2 = LAM_ONE - q0 - q1;
                    if (q2 < 0) {
                        if (q0 >= q1) q0 += q2; else q1 += q2;
                    }
                    l0[i] = q0;
                    l1[i] = q1;
                } else {
                    l0[i] = lam[0];
                    l1[i] = lam[1];
                }
                vr[i] = (R)ur[i];
                vp[i] = (R)up[i];
                vz[i] = (R)uz[i];
                pid[i] = (int32_t)(next_pid + i);
            }
        });
        if (bad[0]) {
            set_error("pic_particles_inject: a particle lies outside the mesh or is not finite");
            return PIC_ERR_ARG;
        }
        if (!have_species) {
            have_species = true;
            q = q_;
            mass = m_;
            weight = w_;
            qm = q_ / m_;
            q_src = qsrc;
        }
        Particles<P> &p = parts[cur];
        PIC_CUDA_TRY(cudaMemcpyAsync(p.tri + n_now, tri.data(), 4 * n, cudaMemcpyHostToDevice, s));
        PIC_CUDA_TRY(cudaMemcpyAsync(p.l0 + n_now, l0.data(), sizeof(Lam) * n, cudaMemcpyHostToDevice, s));
        PIC_CUDA_TRY(cudaMemcpyAsync(p.l1 + n_now, l1.data(), sizeof(Lam) * n, cudaMemcpyHostToDevice, s));
        PIC_CUDA_TRY(cudaMemcpyAsync(p.ur + n_now, vr.data(), sizeof(R) * n, cudaMemcpyHostToDevice, s));
        PIC_CUDA_TRY(cudaMemcpyAsync(p.up + n_now, vp.data(), sizeof(R) * n, cudaMemcpyHostToDevice, s));
        PIC_CUDA_TRY(cudaMemcpyAsync(p.uz + n_now, vz.data(), sizeof(R) * n, cudaMemcpyHostToDevice, s));
        PIC_CUDA_TRY(cudaMemcpyAsync(p.pid + n_now, pid.data(), 4 * n, cudaMemcpyHostToDevice, s));
        int64_t n_new = n_now + n;
        PIC_CUDA_TRY(cudaMemcpyAsync(d_n, &n_new, sizeof(int64_t), cudaMemcpyHostToDevice, s));
        launch_deposit_q<P>(rec, p, n_now, n, Qn(), s);
        n_bound = emitting ? cap : n_new;
        next_pid += n;
        if (emitter_ever) {
            unsigned long long np = (unsigned long long)next_pid;
            PIC_CUDA_TRY(cudaMemcpyAsync(counters + CNT_NEXT_PID, &np, sizeof np, cudaMemcpyHostToDevice, s));
        }
        n_injected += n;
        resort(s);
        PIC_CUDA_TRY(cudaGetLastError());
        PIC_CUDA_TRY(cudaStreamSynchronize(s));
        dgl_dirty = true;
        return PIC_OK;
    }

    void set_graph(bool on) override {
        use_graph = on;
        if (!on && g_exec) {
            cudaGraphExecDestroy(g_exec);
            g_exec = nullptr;
        }
    }

    pic_status step(int64_t n, cudaStream_t s) override {
        if (n < 0) {
            set_error("pic_step: negative step count");
            return PIC_ERR_ARG;
        }
        if (!use_graph || timing_on) return step_direct(n, s);
        const int64_t L = sort_interval > 0 ? 2 * (int64_t)sort_interval : 2;
        int64_t done = 0;
        pic_status st;
        while (done < n) {
            const int64_t left = n - done;
            // a new Gauss-law reference, a first launch (lazy kernel set-up) or a tail
            // shorter than a period: plain steps
            if (dgl_dirty || !stepped || left < L) {
                const int64_t k = (dgl_dirty || !stepped) ? 1 : left;
                if ((st = step_direct(k, s)) != PIC_OK) return st;
                done += k;
                continue;
            }
            // a graph records the launch shapes and the pusher with the buffers
            if (g_exec && (g_bound != n_bound || g_interval != sort_interval || g_ctas != tune_ctas ||
                           g_block != tune_block || g_pusher != pusher || g_src != src_version ||
                           g_wait != wait_polls)) {
                cudaGraphExecDestroy(g_exec);
                g_exec = nullptr;
            }
            if (g_exec && (g_cur != cur || g_qcur != qcur || g_since != since_sort)) {
                // another phase of the period: plain steps until it comes round
                if ((st = step_direct(1, s)) != PIC_OK) return st;
                done += 1;
                continue;
            }
            if (!g_exec && (st = capture(L)) != PIC_OK) return st;
            PIC_CUDA_TRY(cudaGraphLaunch(g_exec, s));
            note_launches(g_kernels);
            n_steps += L;
            done += L;
        }
        return PIC_OK;
    }

    // Launch-shape autotuner.  Coordinate descent over three knobs that change no result
    // (a re-sort only reorders slots, and the kernels' arithmetic does not depend on the
    // grid or the block size): the re-sort interval, the particle kernel's CTAs per SM
    // and the field kernels' block size.  Each trial runs `trial` steps to settle and
    // `trial` timed steps (CUDA events on the stream); the simulation advances through all
    // of them.  Keeps the fastest setting.
    pic_status autotune(int32_t trial, pic_tuning *out, cudaStream_t s) override {
        if (trial < 1) {
            set_error("pic_sim_autotune: trial length must be positive");
            return PIC_ERR_ARG;
        }
        const bool graph = use_graph;
        use_graph = false;
        cudaEvent_t e0, e1;
        PIC_CUDA_TRY(cudaEventCreate(&e0));
        PIC_CUDA_TRY(cudaEventCreate(&e1));
        pic_status st = PIC_OK;
        auto run = [&](double &ms) -> pic_status {
            pic_status r;
            if ((r = step_direct(trial, s)) != PIC_OK) return r;
            PIC_CUDA_TRY(cudaEventRecord(e0, s));
            if ((r = step_direct(trial, s)) != PIC_OK) return r;
            PIC_CUDA_TRY(cudaEventRecord(e1, s));
            PIC_CUDA_TRY(cudaEventSynchronize(e1));
            float x = 0;
            PIC_CUDA_TRY(cudaEventElapsedTime(&x, e0, e1));
            ms = x / trial;
            return PIC_OK;
        };
        double best = 0;
        st = run(best);
        const int32_t sorts[] = {8, 16, 32}, ctas[] = {0, 3, 2}, blocks[] = {128, 256, 512};
        int32_t *knob[] = {&sort_interval, &tune_ctas, &tune_block};
        const int32_t *cand[] = {sorts, ctas, blocks};
        for (int k = 0; k < 3 && st == PIC_OK; k++) {
            const int32_t keep = *knob[k];
            int32_t choice = keep;
            for (int c = 0; c < 3 && st == PIC_OK; c++) {
                if (cand[k][c] == keep) continue;
                *knob[k] = cand[k][c];
                double ms = 0;
                if ((st = run(ms)) == PIC_OK && ms < best) {
                    best = ms;
                    choice = cand[k][c];
                }
            }
            *knob[k] = choice;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        use_graph = graph;
        if (st != PIC_OK) return st;
        if (out) {
            out->sort_interval = sort_interval;
            out->ctas_per_sm = tune_ctas;
            out->field_block = tune_block;
            out->ms_per_step = best;
        }
        return PIC_OK;
    }

    // record one period of steps, from the current phase, into g_exec (nothing runs)
    pic_status capture(int64_t L) {
        if (!g_stream) PIC_CUDA_TRY(cudaStreamCreateWithFlags(&g_stream, cudaStreamNonBlocking));
        const int64_t n0 = n_steps;
        g_cur = cur;
        g_qcur = qcur;
        g_since = since_sort;
        g_bound = n_bound;
        g_interval = sort_interval;
        g_ctas = tune_ctas;
        g_block = tune_block;
        g_pusher = pusher;
        g_wait = wait_polls;
        g_src = src_version;
        PIC_CUDA_TRY(cudaStreamBeginCapture(g_stream, cudaStreamCaptureModeThreadLocal));
        const long long k0 = launches_this_thread();
        pic_status st = step_direct(L, g_stream);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(g_stream, &graph);
        n_steps = n0;
        g_kernels = launches_this_thread() - k0;   // recorded, not run
        note_launches(-g_kernels);
        if (st != PIC_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess) {
            set_error("CUDA error %s: stream capture of the step", cudaGetErrorString(e));
            return PIC_ERR_CUDA;
        }
        e = cudaGraphInstantiate(&g_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            g_exec = nullptr;
            set_error("CUDA error %s: graph instantiation", cudaGetErrorString(e));
            return PIC_ERR_CUDA;
        }
        return PIC_OK;
    }

    // the part of a step before the particle kernel: the Gauss-law reference of a new
    // state, emission, the face kernel (B update, J / Q_abs cleared), probes and ports
    pic_status step_begin(FieldArgs<P> &fa, cudaStream_t s) {
        if (dgl_dirty) {
            // DGL reference res = D_div D^n - Q^n before the first step of this state
            PIC_CUDA_TRY(cudaMemsetAsync(Qwall, 0, sizeof(Acc) * m->N0, s));
            launch_diag<P>(dd, J, Qn(), Qbuf[1 - qcur], Qabs, nullptr, Qwall, D, dgl_ref, 1, E, B, mu_inv,
                           parts[cur], d_n, n_bound, q_scale(), 0.0, diag_out, s);
            dgl_dirty = false;
        }
        if (emitting) {
            EmitArgs<P> ea;
            ea.line = eline;
            ea.p = parts[cur];
            ea.rec = rec;
            ea.n_slots = d_n;
            ea.counters = counters;
            ea.Qn = Qn();
            ea.Qwall = Qwall;
            ea.cap = cap;
            ea.per_step = em.per_step;
            ea.rho0 = em.rho0;
            ea.rho1 = em.rho1;
            ea.u_normal = em.u_normal;
            ea.u_thermal = em.u_thermal;
            ea.seed = (unsigned long long)em.seed;
            launch_emit<P>(ea, s);
        }
        // the face kernel clears J, Q_abs and (FP64) Q^{n+1}; in the FP32 build Q^{n+1} is
        // written whole by the per-node update
        fa.Qn = Qn();
        fa.Qnext = Qbuf[1 - qcur];
        launch_field_b<P>(fa, s);
        if (probes_on) launch_probe<P>(probe, s);
        if (ports_on) launch_port<P>(port, s);
        return PIC_OK;
    }

    // the particle kernel's arguments for the slots `view` (the whole state, or a range of
    // it), counted by the device value at `count`
    PushArgs<P> push_args(const Particles<P> &view, const int64_t *count) const {
        PushArgs<P> pa;
        pa.rec = rec;
        pa.p = view;
        pa.n_slots = count;
        pa.J = J;
        pa.Q = Qbuf[1 - qcur];
        pa.Qabs = Qabs;
        pa.counters = counters;
        pa.qmdt2 = (R)(0.5 * qm * dt);
        pa.dt = (R)dt;
        pa.inv_c2 = (R)(1.0 / (m->units.c * m->units.c));
        pa.bz = (R)bz;
        pa.walk_cap = m->units.walk_cap;
        pa.ctas_per_sm = tune_ctas;
        pa.pusher = pusher;
        pa.wait_polls = wait_polls;
        return pa;
    }

    // the part of a step after the particle kernel: the E update (edge residual, SpMV,
    // node charge), the step count and, when due, the re-sort
    void step_end(FieldArgs<P> &fa, cudaStream_t s) {
        launch_field_e<P>(fa, s);
        qcur = 1 - qcur;
        n_steps++;
        if (sort_interval > 0 && ++since_sort >= sort_interval) resort(s);
    }

    pic_status step_direct(int64_t n, cudaStream_t s) {
        stepped = true;
        FieldArgs<P> fa = field_args();
        for (int64_t it = 0; it < n; it++) {
            pic_status st = step_begin(fa, s);
            if (st != PIC_OK) return st;
            const PushArgs<P> pa = push_args(parts[cur], d_n);
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            if (timing_on) {
                e0 = take_event();
                e1 = take_event();
                cudaEventRecord(e0, s);
            }
            launch_push<P>(pa, n_bound, s);
            if (timing_on) {
                cudaEventRecord(e1, s);
                ev_pending.push_back({e0, e1});
            }
            step_end(fa, s);
        }
        PIC_CUDA_TRY(cudaGetLastError());
        return PIC_OK;
    }

    cudaEvent_t take_event() {
        if (!ev_free.empty()) {
            cudaEvent_t e = ev_free.back();
            ev_free.pop_back();
            return e;
        }
        cudaEvent_t e;
        cudaEventCreate(&e);
        return e;
    }

    pic_status timing(int enable, double *ms, int64_t *launches, cudaStream_t s) override {
        PIC_CUDA_TRY(cudaStreamSynchronize(s));
        double tot = 0;
        for (auto &pr : ev_pending) {
            float x = 0;
            PIC_CUDA_TRY(cudaEventElapsedTime(&x, pr.first, pr.second));
            tot += x;
            ev_free.push_back(pr.first);
            ev_free.push_back(pr.second);
        }
        if (ms) *ms = tot;
        if (launches) *launches = (int64_t)ev_pending.size();
        ev_pending.clear();
        timing_on = enable != 0;
        return PIC_OK;
    }

    pic_status diagnostics(pic_diag *o, double *Eo, double *Bo, double *Jo, cudaStream_t s) override {
        if (dgl_dirty) {
            PIC_CUDA_TRY(cudaMemsetAsync(Qwall, 0, sizeof(Acc) * m->N0, s));
            launch_diag<P>(dd, J, Qn(), Qbuf[1 - qcur], Qabs, nullptr, Qwall, D, dgl_ref, 1, E, B, mu_inv,
                           parts[cur], d_n, n_bound, q_scale(), 0.0, diag_out, s);
            dgl_dirty = false;
        }
        double out[8] = {0};
        unsigned long long cnt[CNT_N] = {0};
        if (o) {
            PIC_CUDA_TRY(cudaMemsetAsync(diag_out, 0, sizeof(double) * 8, s));
            double inv_c2 = 1.0 / (m->units.c * m->units.c);
            Acc *qp = nullptr;
            if constexpr (P::fixed) {
                // Eq. charge evaluated at the current positions, to check the carried Q
                int64_t ns = 0;
                pic_status st = read_count(&ns, s);
                if (st != PIC_OK) return st;
                PIC_CUDA_TRY(cudaMemsetAsync(qpos, 0, sizeof(Acc) * m->N0, s));
                launch_deposit_q<P>(rec, parts[cur], 0, ns, qpos, s);
                qp = qpos;
            }
            // the last step wrote Q^{n+1} into Qn() and kept Q^n in the other buffer
            launch_diag<P>(dd, J, Qn(), Qbuf[1 - qcur], Qabs, qp, Qwall, D, dgl_ref, 0, E, B, mu_inv,
                           parts[cur], d_n, n_bound, q_scale(), inv_c2, diag_out, s);
            PIC_CUDA_TRY(cudaGetLastError());
            PIC_CUDA_TRY(cudaMemcpyAsync(out, diag_out, sizeof out, cudaMemcpyDeviceToHost, s));
            PIC_CUDA_TRY(cudaMemcpyAsync(cnt, counters, sizeof cnt, cudaMemcpyDeviceToHost, s));
        }
        std::vector<R> eh, bh;
        std::vector<double> jd;
        double *jdev = nullptr;
        if (Eo) {
            eh.resize(m->N1);
            PIC_CUDA_TRY(cudaMemcpyAsync(eh.data(), E, sizeof(R) * m->N1, cudaMemcpyDeviceToHost, s));
        }
        if (Bo) {
            bh.resize(m->N2);
            PIC_CUDA_TRY(cudaMemcpyAsync(bh.data(), B, sizeof(R) * m->N2, cudaMemcpyDeviceToHost, s));
        }
        if (Jo) {
            pic_status st = dalloc(jdev, m->N1);
            if (st != PIC_OK) return st;
            launch_acc_to_double<P>(J, jdev, m->N1, j_scale(), s);
            jd.resize(m->N1);
            PIC_CUDA_TRY(cudaMemcpyAsync(jd.data(), jdev, sizeof(double) * m->N1, cudaMemcpyDeviceToHost, s));
        }
        PIC_CUDA_TRY(cudaStreamSynchronize(s));
        if (jdev) release(jdev);
        if (o && cnt[CNT_TIMEOUT]) {
            set_error("pic_diagnostics: %llu bounded device waits timed out; the state is invalid",
                      (unsigned long long)cnt[CNT_TIMEOUT]);
            return PIC_ERR_TIMEOUT;
        }
        if (o) {
            o->n_absorbed = (int64_t)cnt[CNT_ABSORBED];
            o->walk_overflows = (int64_t)cnt[CNT_OVERFLOW];
            o->n_crossings = (int64_t)cnt[CNT_CROSSINGS];
            o->n_particles = n_injected + (int64_t)cnt[CNT_EMITTED] - (int64_t)cnt[CNT_ABSORBED];
            o->n_emitted = (int64_t)cnt[CNT_EMITTED];
            o->emit_dropped = (int64_t)cnt[CNT_EMIT_DROPPED];
            o->steps_since_sort = since_sort;
            o->sort_interval = sort_interval;
            o->n_steps = n_steps;
            o->dce_max = out[0];
            o->dce_nonzero = (int64_t)out[1] + (int64_t)cnt[CNT_REMAINDER];
            o->nr_dce_max = out[2];
            o->dgl_drift = out[3] / (out[4] > 0 ? out[4] : 1.0);
            o->field_energy = out[5];
            o->kinetic_energy = out[6] * mass * weight * m->units.c * m->units.c;
            o->q_absorbed = (double)cnt[CNT_ABSORBED] * q * weight;
        }
        if (Eo)
            for (int64_t i = 0; i < m->N1; i++) Eo[i] = (double)eh[i];
        if (Bo)
            for (int64_t i = 0; i < m->N2; i++) Bo[i] = (double)bh[i];
        if (Jo) std::copy(jd.begin(), jd.end(), Jo);
        return PIC_OK;
    }

    void release(void *p) {
        auto it = std::find(allocs.begin(), allocs.end(), p);
        if (it != allocs.end()) allocs.erase(it);
        if (al.free) al.free(p, al.ctx);
        else cudaFree(p);
    }

    // PIC_ERR_TIMEOUT if a bounded device wait of an earlier step gave up (the state is
    // then invalid); synchronises the stream, allocates nothing
    pic_status waits_ok(const char *who, cudaStream_t s) {
        unsigned long long n = 0;
        PIC_CUDA_TRY(cudaMemcpyAsync(&n, counters + CNT_TIMEOUT, sizeof n, cudaMemcpyDeviceToHost, s));
        PIC_CUDA_TRY(cudaStreamSynchronize(s));
        if (n) {
            set_error("%s: %llu bounded device waits timed out; the state is invalid", who, n);
            return PIC_ERR_TIMEOUT;
        }
        return PIC_OK;
    }

    // pic_charges_get without any allocation: the conversion kernel writes into the
    // library's static scratch, then each part is copied straight into the caller's
    // host array.  Every value of the used part is overwritten, so no clearing is needed.
    pic_status charges_static(double *Qo, double *Qpo, double *Qao, cudaStream_t s) override {
        if (m->N0 > STATIC_MAX_NODES) {
            set_error("pic_charges_get_static: the mesh has %lld nodes, the static scratch "
                      "holds %lld; use pic_charges_get",
                      (long long)m->N0, (long long)STATIC_MAX_NODES);
            return PIC_ERR_ARG;
        }
        pic_status st = waits_ok("pic_charges_get_static", s);
        if (st != PIC_OK) return st;
        double *scr = nullptr;
        st = charge_scratch_address(&scr);
        if (st != PIC_OK) return st;
        const double sc_ = (P::fixed ? LAM_INV : 1.0) * q_src;
        double *outs[3] = {Qo, Qpo, Qao};
        const Acc *ins[3] = {Qn(), Qbuf[1 - qcur], Qabs};
        for (int k = 0; k < 3; k++)
            if (outs[k]) launch_acc_to_double<P>(ins[k], scr + k * m->N0, m->N0, sc_, s);
        PIC_CUDA_TRY(cudaGetLastError());
        for (int k = 0; k < 3; k++)
            if (outs[k])
                PIC_CUDA_TRY(cudaMemcpyAsync(outs[k], scr + k * m->N0, sizeof(double) * m->N0,
                                             cudaMemcpyDeviceToHost, s));
        PIC_CUDA_TRY(cudaStreamSynchronize(s));
        return PIC_OK;
    }

    pic_status charges(double *Qo, double *Qpo, double *Qao, cudaStream_t s) override {
        pic_status st = waits_ok("pic_charges_get", s);
        if (st != PIC_OK) return st;
        double *tmp = nullptr;
        st = dalloc(tmp, 3 * m->N0);
        if (st != PIC_OK) return st;
        double sc_ = (P::fixed ? LAM_INV : 1.0) * q_src;
        launch_acc_to_double<P>(Qn(), tmp, m->N0, sc_, s);
        launch_acc_to_double<P>(Qbuf[1 - qcur], tmp + m->N0, m->N0, sc_, s);
        launch_acc_to_double<P>(Qabs, tmp + 2 * m->N0, m->N0, sc_, s);
        std::vector<double> h(3 * m->N0);
        cudaError_t e = cudaMemcpyAsync(h.data(), tmp, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        release(tmp);
        if (e != cudaSuccess) {
            set_error("pic_charges_get: %s", cudaGetErrorString(e));
            return PIC_ERR_CUDA;
        }
        if (Qo) std::copy(h.begin(), h.begin() + m->N0, Qo);
        if (Qpo) std::copy(h.begin() + m->N0, h.begin() + 2 * m->N0, Qpo);
        if (Qao) std::copy(h.begin() + 2 * m->N0, h.end(), Qao);
        return PIC_OK;
    }

    pic_status count(int64_t *n, cudaStream_t s) override {
        pic_status st = read_count(n, s);
        if (st == PIC_OK && !emitting) n_bound = std::min(n_bound, *n);
        return st;
    }

    pic_status get(int64_t cap_out, int64_t *pid, int32_t *tri, double *lam, double *u,
                   cudaStream_t s) override {
        int64_t n = 0;
        pic_status st = read_count(&n, s);
        if (st != PIC_OK) return st;
        if (n > cap_out) {
            set_error("pic_particles_get: %lld slots exceed the output capacity", (long long)n);
            return PIC_ERR_ARG;
        }
        if (n == 0) return PIC_OK;
        double *lam_d = nullptr, *u_d = nullptr;
        int64_t *pid_d = nullptr;
        if ((st = dalloc(lam_d, 3 * n)) || (st = dalloc(u_d, 3 * n)) || (st = dalloc(pid_d, n))) return st;
        launch_export<P>(parts[cur], n, rec, lam_d, u_d, pid_d, s);
        std::vector<double> hl(3 * n), hu(3 * n);
        std::vector<int64_t> hp(n);
        std::vector<int32_t> ht(n);
        cudaMemcpyAsync(hl.data(), lam_d, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(hu.data(), u_d, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(hp.data(), pid_d, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(ht.data(), parts[cur].tri, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        release(lam_d);
        release(u_d);
        release(pid_d);
        if (e != cudaSuccess) {
            set_error("pic_particles_get: %s", cudaGetErrorString(e));
            return PIC_ERR_CUDA;
        }
        if (pid) std::copy(hp.begin(), hp.end(), pid);
        if (tri) std::copy(ht.begin(), ht.end(), tri);
        if (lam) std::copy(hl.begin(), hl.end(), lam);
        if (u) std::copy(hu.begin(), hu.end(), u);
        return PIC_OK;
    }

    int64_t raw_bytes() const override { return 4 + 2 * (int64_t)sizeof(Lam) + 3 * (int64_t)sizeof(R); }

    pic_status raw_get(void *dst, int64_t n, cudaStream_t s) override {
        if (!dst || n < 0 || n > cap) {
            set_error("pic_particles_raw_get: bad argument");
            return PIC_ERR_ARG;
        }
        return copy_slots(static_cast<char *>(dst), n, 0, n, false, s);
    }

    pic_status raw_set(const void *src, int64_t n, cudaStream_t s) override {
        if (!src || n < 0 || n > cap) {
            set_error("pic_particles_raw_set: bad argument");
            return PIC_ERR_ARG;
        }
        // copy_slots only reads the host buffer on the way up
        pic_status st = copy_slots(const_cast<char *>(static_cast<const char *>(src)), n, 0, n,
                                   true, s);
        if (st != PIC_OK) return st;
        PIC_CUDA_TRY(cudaMemcpyAsync(d_n, &n, sizeof(int64_t), cudaMemcpyHostToDevice, s));
        n_bound = emitting ? cap : n;
        dgl_dirty = true;
        return PIC_OK;
    }

    // slots [c0, c1) of the raw state, host <-> device (one copy per array; array k starts
    // at sum_{j<k} size_j * raw_stride(n) bytes of the host buffer)
    pic_status copy_slots(char *h, int64_t n, int64_t c0, int64_t c1, bool up, cudaStream_t s) {
        const Particles<P> &p = parts[cur];
        void *dev[6] = {p.tri, p.l0, p.l1, p.ur, p.up, p.uz};
        const size_t sz[6] = {4, sizeof(Lam), sizeof(Lam), sizeof(R), sizeof(R), sizeof(R)};
        for (int k = 0; k < 6; k++) {
            char *d = static_cast<char *>(dev[k]) + sz[k] * c0;
            char *hk = h + sz[k] * c0;
            const size_t bytes = sz[k] * (size_t)(c1 - c0);
            if (up) PIC_CUDA_TRY(cudaMemcpyAsync(d, hk, bytes, cudaMemcpyHostToDevice, s));
            else PIC_CUDA_TRY(cudaMemcpyAsync(hk, d, bytes, cudaMemcpyDeviceToHost, s));
            h += sz[k] * raw_stride(n);
        }
        return PIC_OK;
    }

    // one step of step_host with the particle kernel run chunk by chunk between the
    // copies: chunk c is uploaded once the previous step's write-back of it is done,
    // pushed once it has landed, and written back once it is pushed (or, on a re-sort
    // step, once the re-sort is done)
    pic_status step_host_pipelined(char *h, int64_t n, int64_t chunk, cudaStream_t s) {
        pic_status st;
        stepped = true;
        FieldArgs<P> fa = field_args();
        if ((st = step_begin(fa, s)) != PIC_OK) return st;
        k_chunk_counts<<<1, 32, 0, s>>>(d_n, d_chunk_n, chunk, RT_CHUNKS);
        PIC_LAUNCHED();
        const bool resort_due = sort_interval > 0 && since_sort + 1 >= sort_interval;
        for (int c = 0; c < RT_CHUNKS; c++) {
            const int64_t c0 = std::min(n, c * chunk), c1 = std::min(n, c0 + chunk);
            PIC_CUDA_TRY(cudaStreamWaitEvent(up_stream, rt_chunk[c], 0));
            if (c1 > c0 && (st = copy_slots(h, n, c0, c1, true, up_stream)) != PIC_OK) return st;
            PIC_CUDA_TRY(cudaEventRecord(rt_upc[c], up_stream));
            PIC_CUDA_TRY(cudaStreamWaitEvent(s, rt_upc[c], 0));
            if (c1 > c0) {
                Particles<P> v = parts[cur];
                v.tri += c0;
                v.l0 += c0;
                v.l1 += c0;
                v.ur += c0;
                v.up += c0;
                v.uz += c0;
                v.pid += c0;
                launch_push<P>(push_args(v, d_chunk_n + c), c1 - c0, s);
            }
            if (!resort_due) {
                PIC_CUDA_TRY(cudaEventRecord(rt_pushc[c], s));
                PIC_CUDA_TRY(cudaStreamWaitEvent(rt_stream, rt_pushc[c], 0));
                if (c1 > c0 && (st = copy_slots(h, n, c0, c1, false, rt_stream)) != PIC_OK)
                    return st;
                PIC_CUDA_TRY(cudaEventRecord(rt_chunk[c], rt_stream));
            }
        }
        step_end(fa, s);
        if (resort_due) {
            PIC_CUDA_TRY(cudaEventRecord(rt_step, s));
            PIC_CUDA_TRY(cudaStreamWaitEvent(rt_stream, rt_step, 0));
            for (int c = 0; c < RT_CHUNKS; c++) {
                const int64_t c0 = std::min(n, c * chunk), c1 = std::min(n, c0 + chunk);
                if (c1 > c0 && (st = copy_slots(h, n, c0, c1, false, rt_stream)) != PIC_OK)
                    return st;
                PIC_CUDA_TRY(cudaEventRecord(rt_chunk[c], rt_stream));
            }
        }
        PIC_CUDA_TRY(cudaGetLastError());
        return PIC_OK;
    }

    pic_status step_host(void *state, int64_t n, int64_t steps, cudaStream_t s) override {
        if (!state || n < 0 || n > cap || steps < 0) {
            set_error("pic_step_host: bad argument");
            return PIC_ERR_ARG;
        }
        if (emitting) {
            set_error("pic_step_host: the slot count of a host state cannot grow (emitter set)");
            return PIC_ERR_STATE;
        }
        if (!rt_stream) {
            PIC_CUDA_TRY(cudaStreamCreateWithFlags(&rt_stream, cudaStreamNonBlocking));
            PIC_CUDA_TRY(cudaStreamCreateWithFlags(&up_stream, cudaStreamNonBlocking));
            PIC_CUDA_TRY(cudaEventCreateWithFlags(&rt_up, cudaEventDisableTiming));
            for (auto &e : rt_chunk) PIC_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            for (auto &e : rt_upc) PIC_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            for (auto &e : rt_pushc) PIC_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            PIC_CUDA_TRY(cudaEventCreateWithFlags(&rt_step, cudaEventDisableTiming));
            PIC_CUDA_TRY(cudaEventCreateWithFlags(&rt_done, cudaEventDisableTiming));
        }
        char *h = static_cast<char *>(state);
        // chunks of whole particle-kernel tiles (512 slots), so that a chunk's tiles read
        // none of the next chunk's slots
        const int64_t chunk = ((n + RT_CHUNKS - 1) / RT_CHUNKS + 511) / 512 * 512;
        // FP32 build (without kernel timing): after the first step each chunk is pushed as
        // soon as it has landed and written back as soon as it is pushed, so the step's
        // particle work overlaps both copy directions; the E update and any re-sort follow
        // the last chunk (a re-sort moves slots between chunks: then the write-back waits
        // for it)
        const bool pipe = P::fixed && !timing_on;
        pic_status st;
        if (pipe && !d_chunk_n && (st = dalloc(d_chunk_n, RT_CHUNKS)) != PIC_OK) return st;
        // uploads on their own stream, after the caller's earlier work
        PIC_CUDA_TRY(cudaEventRecord(rt_up, s));
        PIC_CUDA_TRY(cudaStreamWaitEvent(up_stream, rt_up, 0));
        for (int64_t k = 0; k < steps; k++) {
            if (k > 0 && pipe) {
                if ((st = step_host_pipelined(h, n, chunk, s)) != PIC_OK) return st;
                continue;
            }
            // upload; chunk c waits only for the previous step's download of chunk c, so the
            // two copy directions overlap
            for (int c = 0; c < RT_CHUNKS; c++) {
                const int64_t c0 = std::min(n, c * chunk), c1 = std::min(n, c0 + chunk);
                if (k > 0) PIC_CUDA_TRY(cudaStreamWaitEvent(up_stream, rt_chunk[c], 0));
                if (c1 > c0 && (st = copy_slots(h, n, c0, c1, true, up_stream)) != PIC_OK)
                    return st;
            }
            PIC_CUDA_TRY(cudaEventRecord(rt_up, up_stream));
            PIC_CUDA_TRY(cudaStreamWaitEvent(s, rt_up, 0));
            if (k == 0) {
                // the caller's state: its slot count, and a new Gauss-law reference
                PIC_CUDA_TRY(cudaMemcpyAsync(d_n, &n, sizeof(int64_t), cudaMemcpyHostToDevice, s));
                n_bound = emitting ? cap : n;
                dgl_dirty = true;
            }
            if ((st = step(1, s)) != PIC_OK) return st;
            PIC_CUDA_TRY(cudaEventRecord(rt_step, s));
            PIC_CUDA_TRY(cudaStreamWaitEvent(rt_stream, rt_step, 0));
            for (int c = 0; c < RT_CHUNKS; c++) {
                const int64_t c0 = std::min(n, c * chunk), c1 = std::min(n, c0 + chunk);
                if (c1 > c0 && (st = copy_slots(h, n, c0, c1, false, rt_stream)) != PIC_OK)
                    return st;
                PIC_CUDA_TRY(cudaEventRecord(rt_chunk[c], rt_stream));
            }
        }
        PIC_CUDA_TRY(cudaEventRecord(rt_done, rt_stream));
        PIC_CUDA_TRY(cudaStreamWaitEvent(s, rt_done, 0));
        return PIC_OK;
    }
};

}  // namespace pic

using namespace pic;

struct pic_sim {
    std::unique_ptr<pic::SimBase> impl;
};

#define SIM_CHECK(s, name)                                   \
    do {                                                     \
        if (!(s) || !(s)->impl) {                            \
            pic::set_error("%s: null simulation", name);     \
            return PIC_ERR_ARG;                              \
        }                                                    \
        cudaError_t e__ = cudaSetDevice((s)->impl->device);  \
        if (e__ != cudaSuccess) {                            \
            pic::set_error("%s: %s", name, cudaGetErrorString(e__)); \
            return PIC_ERR_CUDA;                             \
        }                                                    \
    } while (0)

extern "C" pic_status pic_set_allocator(pic_alloc_fn alloc, pic_free_fn free_, void *ctx) try {
    if ((alloc == nullptr) != (free_ == nullptr)) {
        set_error("pic_set_allocator: give both functions or neither");
        return PIC_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(g_allocator_mu);
    g_allocator.alloc = alloc;
    g_allocator.free = free_;
    g_allocator.ctx = ctx;
    return PIC_OK;
}
PIC_CATCH("pic_set_allocator")

extern "C" pic_status pic_sim_create(pic_mesh *pm, double dt, double bz, int64_t max_particles,
                                     pic_sim **out) try {
    if (!pm || !out || !(dt > 0) || !std::isfinite(bz) || max_particles < 0 ||
        max_particles >= ((int64_t)1 << 31)) {
        set_error("pic_sim_create: bad argument");
        return PIC_ERR_ARG;
    }
    if (!pm->h.have_spai) {
        set_error("pic_sim_create: call pic_spai_build first");
        return PIC_ERR_STATE;
    }
    if (dt > pm->h.dt_stable) {
        set_error("pic_sim_create: dt %g above the stable limit %g", dt, pm->h.dt_stable);
        return PIC_ERR_UNSTABLE;
    }
    std::unique_ptr<pic_sim> s(new (std::nothrow) pic_sim);
    if (!s) {
        set_error("pic_sim_create: out of host memory");
        return PIC_ERR_OOM;
    }
    pic_status st;
    Allocator al;
    {
        std::lock_guard<std::mutex> lk(g_allocator_mu);
        al = g_allocator;
    }
    if (pm->h.units.precision == PIC_FP32) {
        auto *x = new SimImpl<PF32>;
        x->al = al;
        s->impl.reset(x);
        st = x->init(pm->h, dt, bz, max_particles);
    } else {
        auto *x = new SimImpl<PF64>;
        x->al = al;
        s->impl.reset(x);
        st = x->init(pm->h, dt, bz, max_particles);
    }
    if (st != PIC_OK) return st;
    *out = s.release();
    return PIC_OK;
}
PIC_CATCH("pic_sim_create")

extern "C" pic_status pic_sim_autotune(pic_sim *s, int32_t trial_steps, pic_tuning *out,
                                       void *st) try {
    SIM_CHECK(s, "pic_sim_autotune");
    return s->impl->autotune(trial_steps, out, (cudaStream_t)st);
}
PIC_CATCH("pic_sim_autotune")

extern "C" pic_status pic_sim_set_graph(pic_sim *s, int32_t enable) try {
    SIM_CHECK(s, "pic_sim_set_graph");
    s->impl->set_graph(enable != 0);
    return PIC_OK;
}
PIC_CATCH("pic_sim_set_graph")

extern "C" pic_status pic_sim_set_sort_interval(pic_sim *s, int32_t interval) try {
    SIM_CHECK(s, "pic_sim_set_sort_interval");
    if (interval < 0) {
        set_error("pic_sim_set_sort_interval: negative interval");
        return PIC_ERR_ARG;
    }
    s->impl->sort_interval = interval;
    return PIC_OK;
}
PIC_CATCH("pic_sim_set_sort_interval")

extern "C" pic_status pic_sim_set_pusher(pic_sim *s, int32_t pusher) try {
    SIM_CHECK(s, "pic_sim_set_pusher");
    if (pusher != PIC_PUSHER_BORIS && pusher != PIC_PUSHER_VAY) {
        set_error("pic_sim_set_pusher: unknown pusher %d", (int)pusher);
        return PIC_ERR_ARG;
    }
    s->impl->pusher = pusher;
    return PIC_OK;
}
PIC_CATCH("pic_sim_set_pusher")

extern "C" pic_status pic_launch_count(int64_t *out) try {
    if (!out) {
        set_error("pic_launch_count: null output");
        return PIC_ERR_ARG;
    }
    *out = (int64_t)g_launches.load();
    return PIC_OK;
}
PIC_CATCH("pic_launch_count")

extern "C" pic_status pic_sim_set_wait_limit(pic_sim *s, int64_t polls) try {
    SIM_CHECK(s, "pic_sim_set_wait_limit");
    if (polls < 0) {
        set_error("pic_sim_set_wait_limit: negative poll count");
        return PIC_ERR_ARG;
    }
    s->impl->wait_polls = polls;
    return PIC_OK;
}
PIC_CATCH("pic_sim_set_wait_limit")

extern "C" pic_status pic_sim_set_static_field(pic_sim *s, const double *E_static, void *st) try {
    SIM_CHECK(s, "pic_sim_set_static_field");
    return s->impl->set_static_field(E_static, (cudaStream_t)st);
}
PIC_CATCH("pic_sim_set_static_field")

extern "C" pic_status pic_sim_set_emitter(pic_sim *s, const pic_emitter *e, void *st) try {
    SIM_CHECK(s, "pic_sim_set_emitter");
    return s->impl->set_emitter(e, (cudaStream_t)st);
}
PIC_CATCH("pic_sim_set_emitter")

extern "C" pic_status pic_sim_set_loss(pic_sim *s, const double *sigma_e, const double *sigma_m,
                                       void *st) try {
    SIM_CHECK(s, "pic_sim_set_loss");
    return s->impl->set_loss(sigma_e, sigma_m, (cudaStream_t)st);
}
PIC_CATCH("pic_sim_set_loss")

extern "C" pic_status pic_sim_set_probes(pic_sim *s, int64_t n_entries, const int32_t *face,
                                         const int32_t *group, const double *weight,
                                         int32_t n_groups, const int32_t *power,
                                         int64_t capacity, int32_t every, void *st) try {
    SIM_CHECK(s, "pic_sim_set_probes");
    return s->impl->set_probes(n_entries, face, group, weight, n_groups, power, capacity, every,
                               (cudaStream_t)st);
}
PIC_CATCH("pic_sim_set_probes")

extern "C" pic_status pic_probes_read(pic_sim *s, double *out, int64_t cap_records,
                                      int64_t *n_records, int64_t *n_dropped, void *st) try {
    SIM_CHECK(s, "pic_probes_read");
    return s->impl->probes_read(out, cap_records, n_records, n_dropped, (cudaStream_t)st);
}
PIC_CATCH("pic_probes_read")

extern "C" pic_status pic_sim_set_ports(pic_sim *s, int32_t n_ports, const double *z,
                                        const double *rho0, const double *rho1, int64_t capacity,
                                        int32_t every, void *st) try {
    SIM_CHECK(s, "pic_sim_set_ports");
    return s->impl->set_ports(n_ports, z, rho0, rho1, capacity, every, (cudaStream_t)st);
}
PIC_CATCH("pic_sim_set_ports")

extern "C" pic_status pic_ports_read(pic_sim *s, double *out, int64_t cap_records,
                                     int64_t *n_records, int64_t *n_dropped, void *st) try {
    SIM_CHECK(s, "pic_ports_read");
    return s->impl->ports_read(out, cap_records, n_records, n_dropped, (cudaStream_t)st);
}
PIC_CATCH("pic_ports_read")

extern "C" pic_status pic_fields_set(pic_sim *s, const double *E, const double *B, void *st) try {
    SIM_CHECK(s, "pic_fields_set");
    return s->impl->fields_set(E, B, (cudaStream_t)st);
}
PIC_CATCH("pic_fields_set")

extern "C" pic_status pic_particles_inject(pic_sim *s, int64_t n, const double *z,
                                           const double *rho, const double *ur, const double *up,
                                           const double *uz, double q, double m, double w, void *st) try {
    SIM_CHECK(s, "pic_particles_inject");
    return s->impl->inject(n, z, rho, ur, up, uz, q, m, w, (cudaStream_t)st);
}
PIC_CATCH("pic_particles_inject")

extern "C" pic_status pic_step(pic_sim *s, int64_t n, void *st) try {
    SIM_CHECK(s, "pic_step");
    return s->impl->step(n, (cudaStream_t)st);
}
PIC_CATCH("pic_step")

extern "C" pic_status pic_diagnostics(pic_sim *s, pic_diag *o, double *E, double *B, double *J,
                                      void *st) try {
    SIM_CHECK(s, "pic_diagnostics");
    return s->impl->diagnostics(o, E, B, J, (cudaStream_t)st);
}
PIC_CATCH("pic_diagnostics")

extern "C" pic_status pic_charges_get_static(pic_sim *s, double *Q, double *Qp, double *Qa,
                                             void *st) try {
    SIM_CHECK(s, "pic_charges_get_static");
    return s->impl->charges_static(Q, Qp, Qa, (cudaStream_t)st);
}
PIC_CATCH("pic_charges_get_static")

extern "C" pic_status pic_charges_get(pic_sim *s, double *Q, double *Qp, double *Qa, void *st) try {
    SIM_CHECK(s, "pic_charges_get");
    return s->impl->charges(Q, Qp, Qa, (cudaStream_t)st);
}
PIC_CATCH("pic_charges_get")

extern "C" pic_status pic_particles_count(pic_sim *s, int64_t *n, void *st) try {
    SIM_CHECK(s, "pic_particles_count");
    if (!n) {
        set_error("pic_particles_count: null output");
        return PIC_ERR_ARG;
    }
    return s->impl->count(n, (cudaStream_t)st);
}
PIC_CATCH("pic_particles_count")

extern "C" pic_status pic_particles_get(pic_sim *s, int64_t cap, int64_t *pid, int32_t *tri,
                                        double *lam, double *u, void *st) try {
    SIM_CHECK(s, "pic_particles_get");
    return s->impl->get(cap, pid, tri, lam, u, (cudaStream_t)st);
}
PIC_CATCH("pic_particles_get")

extern "C" pic_status pic_particles_raw_bytes(pic_sim *s, int64_t *b) try {
    SIM_CHECK(s, "pic_particles_raw_bytes");
    if (!b) {
        set_error("pic_particles_raw_bytes: null output");
        return PIC_ERR_ARG;
    }
    *b = s->impl->raw_bytes();
    return PIC_OK;
}
PIC_CATCH("pic_particles_raw_bytes")

extern "C" pic_status pic_particles_raw_size(pic_sim *s, int64_t n_slots, int64_t *bytes) try {
    SIM_CHECK(s, "pic_particles_raw_size");
    if (!bytes || n_slots < 0) {
        set_error("pic_particles_raw_size: bad argument");
        return PIC_ERR_ARG;
    }
    *bytes = SimBase::raw_stride(n_slots) * s->impl->raw_bytes();
    return PIC_OK;
}
PIC_CATCH("pic_particles_raw_size")

extern "C" pic_status pic_particles_raw_get(pic_sim *s, void *dst, int64_t n, void *st) try {
    SIM_CHECK(s, "pic_particles_raw_get");
    return s->impl->raw_get(dst, n, (cudaStream_t)st);
}
PIC_CATCH("pic_particles_raw_get")

extern "C" pic_status pic_particles_raw_set(pic_sim *s, const void *src, int64_t n, void *st) try {
    SIM_CHECK(s, "pic_particles_raw_set");
    return s->impl->raw_set(src, n, (cudaStream_t)st);
}
PIC_CATCH("pic_particles_raw_set")

extern "C" pic_status pic_step_host(pic_sim *s, void *state, int64_t n_slots, int64_t n_steps,
                                     void *st) try {
    SIM_CHECK(s, "pic_step_host");
    return s->impl->step_host(state, n_slots, n_steps, (cudaStream_t)st);
}
PIC_CATCH("pic_step_host")

extern "C" pic_status pic_kernel_timing(pic_sim *s, int32_t enable, double *ms, int64_t *launches,
                                        void *st) try {
    SIM_CHECK(s, "pic_kernel_timing");
    return s->impl->timing(enable, ms, launches, (cudaStream_t)st);
}
PIC_CATCH("pic_kernel_timing")

extern "C" void pic_sim_destroy(pic_sim *s) { delete s; }
