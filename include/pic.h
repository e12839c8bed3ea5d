/*
 * pic.h -- C ABI of the GB300 library for the axisymmetric charge-conservative
 * electromagnetic particle-in-cell method on unstructured triangle meshes of the
 * meridian (z, rho) plane (Na, Omelchenko, Moon, Borges, Teixeira, 2017).
 *
 * One simulation advances, per call of pic_step, the paper's cycle (Sec. 3):
 *   B^{n+1/2} = B^{n-1/2} - dt D_curl E^n                                (Eq. full_d_dfl)
 *   gather E^n and (B^{n+1/2}+B^{n-1/2})/2 at each particle by Whitney forms (Sec. 3.2),
 *   relativistic Boris push (Eqs. DNE, DLE), triangle walk, charge-conserving scatter of
 *   edge currents J^{n+1/2} (Eq. current) and node charges Q^{n+1} (Eq. charge),
 *   E^{n+1} = E^n + dt M (D_curl^T star_mu^-1 B^{n+1/2} - J^{n+1/2})      (Eq. full_d_dal)
 * with M the sparse approximate inverse (SPAI) of the rho-weighted Hodge matrix star_eps.
 *
 * Conventions shared by every call:
 *  - Every call returns a pic_status and never aborts the process.  On an error nothing
 *    is written to the caller's output arrays and pic_last_error() returns a message
 *    (thread-local, valid until the next failing call on the same thread).
 *  - Handles are owned by the library and released by the matching *_destroy call.
 *  - Input arrays are caller-owned host arrays; the library copies what it keeps.
 *  - Output arrays are caller-owned host arrays of the stated size, unless stated.
 *  - Units are the caller's, consistent with eps0, mu0 and c in pic_units.
 *  - Mesh coordinates: nodes are (z, rho) pairs with rho >= 0.  Triangles are node
 *    triples, any orientation (stored counter-clockwise in (z, rho)).  Edges are
 *    oriented from the lower to the higher node index (App. D) and numbered in
 *    lexicographic order of (lower, higher) node index; faces keep the input order.
 *  - Field degrees of freedom: E_e is the line integral of E along edge e (Whitney
 *    1-form), B_f the flux of B_phi through face f (Whitney 2-form, B_phi = B_f / A_f).
 *  - Device memory comes from the allocator installed by pic_set_allocator, or from
 *    cudaMalloc when none is installed.  All device work of a call is ordered on the
 *    stream passed to it (NULL: the legacy default stream).
 */
#ifndef PIC_H
#define PIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pic_mesh pic_mesh; /* opaque: mesh, incidence, Hodge and SPAI operators */
typedef struct pic_sim pic_sim;   /* opaque: device-resident fields and particles      */

typedef enum {
    PIC_OK = 0,
    PIC_ERR_ARG = 1,      /* bad argument (null pointer, size, value out of range)       */
    PIC_ERR_MESH = 2,     /* inconsistent mesh (degenerate triangle, bad boundary list)  */
    PIC_ERR_CUDA = 3,     /* a CUDA runtime call failed                                  */
    PIC_ERR_UNSTABLE = 4, /* dt above the stable leapfrog limit                          */
    PIC_ERR_TIMEOUT = 5,  /* a bounded device wait gave up                               */
    PIC_ERR_OOM = 6,      /* device or host allocation failed / capacity exceeded        */
    PIC_ERR_STATE = 7     /* call out of order (e.g. pic_sim_create before SPAI)         */
} pic_status;

/* boundary tags of mesh boundary edges */
enum {
    PIC_BC_PEC = 1,   /* conductor: tangential E = 0 (edge DOF removed), particles absorbed */
    PIC_BC_AXIS = 2,  /* rho = 0: natural (PMC) field condition, particles stay (Sec. 5.1)  */
    PIC_BC_ABSORB = 3 /* open port: natural field condition, particles absorbed             */
};

/* arithmetic of the particle loop and fields */
enum {
    PIC_FP64 = 0, /* FP64 fields and particles, FP64 atomics for J and Q                   */
    PIC_FP32 = 1  /* FP32 fields and momenta; positions as fixed-point barycentric
                     coordinates (2^-22); J and Q as int64 fixed point (2^-44, 2^-22),
                     so the scatter sums are exact and independent of order             */
};

typedef struct {
    double eps0;       /* vacuum permittivity                                       */
    double mu0;        /* vacuum permeability                                       */
    double c;          /* speed of light (used in gamma = sqrt(1 + |u|^2/c^2))      */
    int32_t precision; /* PIC_FP64 or PIC_FP32                                      */
    int32_t walk_cap;  /* edge crossings per particle per step before the particle
                          is removed and counted as a walk overflow; 0 means 16,
                          at most PIC_WALK_CAP_MAX (bounds every walk loop)         */
} pic_units;

#define PIC_WALK_CAP_MAX 4096

typedef struct {
    int64_t n_particles;     /* live particles                                          */
    int64_t n_absorbed;      /* particles removed at walls since creation                */
    int64_t walk_overflows;  /* particles removed by the walk cap since creation         */
    int64_t n_crossings;     /* edge crossings since creation                            */
    int64_t n_steps;         /* steps taken                                              */
    double dce_max;          /* max over nodes of |(Q^{n+1}-Q^n+Qabs)/dt + D_div J| of the
                                last step, in units of q_src/dt (Eq. DCE)                 */
    int64_t dce_nonzero;     /* FP32: nodes where the fixed-point DCE is not exactly 0  */
    double nr_dce_max;       /* max |NR_DCE| of Sec. 5.1.1 over nodes with net current   */
    double dgl_drift;        /* max over non-PEC nodes of |res^n - res^ref - Q_wall|,
                                res^n = D_div D^n - Q^n (Eq. DGL_RSD_REL), relative to
                                max|Q|; res^ref is taken at the first step after the host
                                last changed fields or particles, and Q_wall is the charge
                                removed at walls since then (it leaves Q without crossing
                                an edge, so it shifts res by exactly that amount)         */
    double field_energy;     /* 1/2 E.star_eps.E + 1/2 B.star_mu^-1.B (per radian)        */
    double kinetic_energy;   /* sum (gamma-1) m c^2 w over live particles (3D)             */
    double q_absorbed;       /* charge removed at walls since creation (3D, q*w units)   */
    int64_t n_emitted;       /* particles born by the emitter since creation              */
    int64_t emit_dropped;    /* particles the emitter did not make for lack of capacity   */
    int64_t steps_since_sort;/* steps since the last re-sort by triangle (the next one
                                comes after the step that makes this sort_interval)     */
    int64_t sort_interval;   /* steps between re-sorts now in force (0: never)          */
} pic_diag;

/* Allocator hook for device memory (e.g. a framework's caching allocator).  alloc must
 * return device memory of at least `bytes` bytes aligned to 256 bytes, or NULL; free
 * releases it.  Install before creating simulations (each keeps the hooks it was created
 * with); pass NULLs to restore cudaMalloc.  Not an operation of the paper.  Errors: ARG
 * (one function given without the other). */
typedef void *(*pic_alloc_fn)(size_t bytes, void *ctx);
typedef void (*pic_free_fn)(void *ptr, void *ctx);
pic_status pic_set_allocator(pic_alloc_fn alloc, pic_free_fn free_, void *ctx);

/* Mesh of the meridian plane (Sec. 3.1, App. D).  nodes_zr: n_nodes x 2 doubles (z, rho);
 * tris: n_tris x 3 node indices; bedge_nodes: n_bedges x 2 node indices, one row per
 * boundary edge of the mesh (every edge with one triangle must be listed exactly once);
 * bedge_tag: PIC_BC_* per boundary edge.  Builds the incidence matrices D_curl (N2 x N1)
 * and D_div (N0 x N1), per-triangle geometry, the rho-weighted Hodge matrix star_eps
 * (Eq. dis_hodge_eps, App. B; exact integration) and the diagonal star_mu^-1
 * (Eq. dis_hodge_mu: rho_bar_f / (mu0 A_f)).  Host-only; no device memory yet.
 * The mesh must be conforming: an edge belongs to one or two triangles, and two triangles
 * sharing an edge lie on opposite sides of it (either node order is accepted per triangle).
 * Errors: PIC_ERR_ARG (null / non-positive sizes / rho < 0 / bad index), PIC_ERR_MESH
 * (degenerate or overlapping triangles, an edge in three triangles, bad boundary list). */
pic_status pic_mesh_create(const double *nodes_zr, int64_t n_nodes, const int32_t *tris,
                           int64_t n_tris, const int32_t *bedge_nodes,
                           const int32_t *bedge_tag, int64_t n_bedges, const pic_units *u,
                           pic_mesh **out);

/* Sizes: nodes N0, edges N1, faces N2, free (non-PEC) edges, nonzeros of M (0 before
 * pic_spai_build).  Any output pointer may be NULL.  Host-only.  Errors: ARG (null mesh). */
pic_status pic_mesh_info(const pic_mesh *m, int64_t *n_nodes, int64_t *n_edges,
                         int64_t *n_tris, int64_t *n_free_edges, int64_t *spai_nnz);

/* Edge list in library numbering (App. D: tail = lower node index): n_edges x 2 node
 * indices (tail, head) into a caller-owned array.  Host-only.  Errors: ARG (null). */
pic_status pic_mesh_edges(const pic_mesh *m, int32_t *edge_nodes);

/* SPAI of star_eps (Sec. 3.1: the explicit, local E update).  Column j of M minimises
 * ||star_eps m - e_j||_2 over vectors supported on the free edges within
 * `pattern_level` triangle-hops of edge j (a dense least-squares problem over the rows
 * those columns touch); entries below drop_tol * max_i |m_i| are dropped and
 * M <- (M + M^T)/2.  Then the stable step dt_max = 2 / sqrt(lambda_max(M K)),
 * K = D_curl^T star_mu^-1 D_curl, by 500 power iterations, is written to *dt_stable_out
 * (may be NULL).  pattern_level in [0, 8], drop_tol in [0, 1).  Host-only. */
pic_status pic_spai_build(pic_mesh *m, int32_t pattern_level, double drop_tol,
                          double *dt_stable_out);

/* Optional: export the free-edge numbering and M in CSR (free-edge indices), into
 * caller-owned arrays sized by pic_mesh_info.  free_edges: n_free entries (may be NULL);
 * indptr: n_free+1; indices, values: nnz.  Host-only.  Errors: ARG, STATE (no SPAI). */
pic_status pic_spai_get(const pic_mesh *m, int32_t *free_edges, int64_t *indptr,
                        int32_t *indices, double *values);

/* Quality of the SPAI (Sec. 3.1; not an operation of the paper): nnz of M, and the
 * residual R = star_eps_ff M - I over the free edges, as ||R||_F / sqrt(n_free) (the RMS
 * of the per-column residual norms) and max |R_ij|.  Host-only; each output may be NULL.
 * Errors: STATE (no SPAI built). */
pic_status pic_spai_info(const pic_mesh *m, int64_t *nnz, double *residual_rms,
                         double *residual_max);

/* Simulation on the current CUDA device: uploads the mesh operators and allocates
 * fields and room for `max_particles` particles.  dt must not exceed the stable step
 * from pic_spai_build (PIC_ERR_UNSTABLE otherwise); bz_guide is a uniform static axial
 * magnetic field added at the gather (Sec. 3.2, beam focusing system).  The mesh must
 * outlive the simulation.  Fields start at zero.  Errors: ARG, STATE (no SPAI), UNSTABLE,
 * OOM, CUDA. */
pic_status pic_sim_create(pic_mesh *m, double dt, double bz_guide, int64_t max_particles,
                          pic_sim **out);

/* Steps between particle re-sorts by triangle (default 16; 0 disables re-sorting).  Not
 * an operation of the paper: it keeps the particles of a triangle together in memory.
 * Errors: ARG (null handle, negative interval). */
pic_status pic_sim_set_sort_interval(pic_sim *s, int32_t interval);

/* Velocity update of Eq. DLE (Sec. 3.3 adopts a corrected Boris scheme, citing Vay 2008).
 * PIC_PUSHER_BORIS (default): half electric kick, rotation by the angle of
 * t = q dt B / (2 m gamma(u-)), half electric kick; the magnetic term of Eq. DLE then
 * uses the mean of u^{n-1/2} and u^{n+1/2} with one gamma.  PIC_PUSHER_VAY: the magnetic
 * term uses the mean of the velocities v^{n-1/2} and v^{n+1/2}, and Eq. DLE is solved for
 * u^{n+1/2} in closed form (gamma^{n+1/2} from a quadratic in gamma^2), which keeps a
 * particle in crossed fields with E + v x B = 0 unaccelerated.  Both build precisions.
 * Errors: ARG (null handle or unknown pusher). */
enum { PIC_PUSHER_BORIS = 0, PIC_PUSHER_VAY = 1 };
pic_status pic_sim_set_pusher(pic_sim *s, int32_t pusher);

/* Bound of the particle kernel's tile-pipeline waits (FP32 build): the number of polls,
 * each suspending the waiting thread for at most 100 us, that a wait for a staged tile
 * (or for the release of a buffer) makes before it gives up.  Default 16384 (about 1.6 s).
 * A wait that gives up is counted on the device; the block then stops, and before it
 * exits it waits, with the default bound, for every copy into its shared memory still in
 * flight, so a give-up never leaves a copy running.  Not an operation of the paper: it
 * lets a caller (a test) make the waits run out, with 0 polls, and see the step reported
 * as PIC_ERR_TIMEOUT by the next pic_diagnostics, pic_charges_get or
 * pic_charges_get_static.  The simulation's state is invalid after that.
 * Errors: ARG (null handle, negative count). */
pic_status pic_sim_set_wait_limit(pic_sim *s, int64_t polls);

/* Sources either side of the particle loop (Secs. 5.2, 5.3).
 *
 * The static (gun) field of the electrodes, by Poisson's equation (Sec. 5.3): the node
 * potential phi with phi held at held_nodes (n_held of them, potentials held_phi) and
 * D_div star_eps D_div^T phi = Q at every other node, i.e. the discrete Gauss law for
 * E = -grad phi, whose Whitney-1 edge values are phi(tail) - phi(head) (zero normal flux
 * where no potential is held).  charge: node charges Q (N0, per radian like star_eps:
 * w q / (2 pi) per unit barycentric weight), or NULL for none.  Solved on the host by
 * conjugate gradients; phi_out (N0) and E_out (N1) may each be NULL.  Errors: ARG, MESH
 * (a part of the mesh reaches no held node). */
pic_status pic_static_potential(const pic_mesh *m, int64_t n_held, const int32_t *held_nodes,
                                const double *held_phi, const double *charge, double *phi_out,
                                double *E_out);

/* A static field (N1 edge values, e.g. E_out above) added to E^n at the gather only: it
 * drives the particles but takes no part in the leapfrog (the electrodes' voltage is held
 * by it, the self-field sees grounded conductors).  NULL removes it.  Copied; synchronous.
 * Errors: ARG (not finite), OOM, CUDA. */
pic_status pic_sim_set_static_field(pic_sim *s, const double *E_static, void *cuda_stream);

/* Emission: at the start of every step, before the particle kernel, per_step particles
 * are born on the line z = z (inside the mesh, crossing no node), rho uniform in area over
 * [rho0, rho1]; momenta u = gamma v with independent normal components of standard
 * deviation u_thermal about (0, 0, u_normal).  Their charge is added to Q^n at the birth
 * point (Eq. charge), so Eq. DCE holds for the step, and is taken out of the Gauss-law
 * drift.  Draws are counter-based: for particle id p and draw j (0: rho, 1-2 and 3-4:
 * Box-Muller pairs), splitmix64(seed + 8 p + j) >> 11 as (k + 1/2) 2^-53.  Particle ids
 * continue the count of all particles made.  A step whose births do not fit the capacity
 * makes none (counted in pic_diag.emit_dropped).  One species per simulation (q/m and
 * q*w as for pic_particles_inject).  While an emitter is set, launches are sized for the
 * capacity.  NULL stops emission.  Not in the paper's equations: the paper injects at
 * the cathode without giving the distribution.  Errors: ARG, OOM, CUDA. */
typedef struct {
    double z;          /* emission line z = const                                   */
    double rho0, rho1; /* radial extent                                             */
    int64_t per_step;  /* particles born per step                                   */
    double u_normal;   /* mean u_z of the new particles                             */
    double u_thermal;  /* standard deviation of each momentum component             */
    uint64_t seed;     /* generator key                                             */
    double q, m, w;    /* species: charge, mass, macro-particle weight              */
} pic_emitter;
pic_status pic_sim_set_emitter(pic_sim *s, const pic_emitter *e, void *cuda_stream);

/* Absorbing layer (the paper ends its ports and left walls with a PML, Sec. 5.3, without
 * giving its equations; this is a documented substitute): electric conductivity sigma_e
 * per edge (N1, S/m) and magnetic conductivity sigma_m per face (N2, ohm/m), both >= 0,
 * e.g. graded from 0 at the layer's inner face, sigma_m = sigma_e mu0 / eps0 for a
 * matched layer.  With s = sigma_e dt / (2 eps0) the E update of Eq. full_d_dal becomes
 * E <- (1 - s)/(1 + s) E + dt (M r) / (1 + s) on each free edge, and with
 * s = sigma_m dt / (2 mu0) Eq. full_d_dfl becomes B <- (1 - s)/(1 + s) B - dt D_curl E
 * / (1 + s) on each face (the conduction terms time-centred).  Conduction moves charge in
 * the layer, so its nodes leave the Gauss-law drift (a new reference is taken).  Both
 * NULL: lossless.  Copied; synchronous.  Errors: ARG (negative or not finite), OOM, CUDA. */
pic_status pic_sim_set_loss(pic_sim *s, const double *sigma_e, const double *sigma_m,
                            void *cuda_stream);

/* Field probes recorded on the device (field values and energy envelopes): n_entries (face, group, weight) triples; after the B update of a step,
 * group g sums weight * B_f (power[g] = 1) or weight * B_f^2 (power[g] = 2) over its
 * entries, B being B^{n+1/2}.  Every `every` steps, counted from this call, the n_groups
 * sums are appended to a device buffer of `capacity` records; nothing else waits for the
 * host.  n_entries = 0 removes the probes.  Device memory of earlier probe sets is held
 * until the simulation is destroyed.  Errors: ARG, OOM, CUDA.  Not an operation of the
 * paper. */
pic_status pic_sim_set_probes(pic_sim *s, int64_t n_entries, const int32_t *face,
                              const int32_t *group, const double *weight, int32_t n_groups,
                              const int32_t *power, int64_t capacity, int32_t every,
                              void *cuda_stream);

/* Copy out the records made since the last read (at most cap_records x n_groups doubles,
 * record-major) and start a new set; *n_dropped counts records that found the buffer full
 * or did not fit cap_records.  Synchronous.  Errors: STATE (no probes), CUDA. */
pic_status pic_probes_read(pic_sim *s, double *out, int64_t cap_records, int64_t *n_records,
                           int64_t *n_dropped, void *cuda_stream);

/* Output-port signal recorded on the device: the BWO's output power (Secs. 5.1, 5.1.1),
 * as the Poynting flux through planes z = z[k], rho0[k] <= rho <= rho1[k]:
 *   P_k = (2 pi / mu0) int_rho0^rho1 E_rho B_phi rho drho,
 * with E^n (Whitney 1-form, the static field included when one is set) and the
 * time-centred B_phi = (B^{n+1/2} + B^{n-1/2}) / (2 A) (Whitney 2-form) of step n, the
 * fields the gather of that step sees.  Each plane is cut into the chords of the triangles
 * it crosses; E_rho and rho are linear along a chord and B_phi is constant, so two
 * Gauss-Legendre points per chord give the integral of the discrete fields exactly.
 * Positive P flows toward +z.  Every `every` steps, counted from this call, the n_ports
 * values are appended to a device buffer of `capacity` records (nothing waits for the
 * host; graph replay records too).  n_ports = 0 removes the ports.  Errors: ARG (a plane
 * that does not cross the mesh in one piece between rho0 and rho1, or passes through a
 * node; bad sizes), OOM, CUDA.  Units: watts for SI fields. */
pic_status pic_sim_set_ports(pic_sim *s, int32_t n_ports, const double *z, const double *rho0,
                             const double *rho1, int64_t capacity, int32_t every,
                             void *cuda_stream);

/* Copy out the port records made since the last read (at most cap_records x n_ports
 * doubles, record-major) and start a new set; as pic_probes_read.  Errors: STATE (no
 * ports), CUDA. */
pic_status pic_ports_read(pic_sim *s, double *out, int64_t cap_records, int64_t *n_records,
                          int64_t *n_dropped, void *cuda_stream);

/* Replay steps from a CUDA graph (off by default).  pic_step then records one period of
 * 2 x the re-sort interval steps (2 with re-sorting off) on an internal stream the first
 * time it is needed, and launches that graph on the caller's stream for every whole period
 * that starts at the recorded phase; other steps run as before.  Results are those of plain
 * steps.  The graph is recorded again after the slot bound, the re-sort interval, the
 * launch shapes or the pusher changed;
 * per-launch timing (pic_kernel_timing) bypasses it.  Not an operation of the paper: it
 * removes the host launch cost of small meshes. */
pic_status pic_sim_set_graph(pic_sim *s, int32_t enable);

/* Launch shapes picked by pic_sim_autotune (not an operation of the paper). */
typedef struct {
    int32_t sort_interval;  /* steps between re-sorts by triangle                        */
    int32_t ctas_per_sm;    /* persistent CTAs per SM of the particle kernel (0: all fit) */
    int32_t field_block;    /* threads per block of the field kernels                    */
    int32_t pad;
    double ms_per_step;     /* device time per step of the chosen setting                */
} pic_tuning;

/* Autotuner: coordinate descent over the re-sort interval (8, 16, 32), the particle
 * kernel's CTAs per SM (all that fit, 3, 2) and the field kernels' block size (128, 256,
 * 512), none of which changes a result (the FP32 state after tuning is bit for bit that
 * of the same number of plain steps).  Each trial runs trial_steps steps to settle and
 * trial_steps timed steps: the simulation advances by up to 14 x trial_steps steps.  The
 * fastest setting stays in effect and is written to *out (may be NULL).  Synchronous.
 * Errors: PIC_ERR_ARG (trial_steps < 1), CUDA errors of the steps. */
pic_status pic_sim_autotune(pic_sim *s, int32_t trial_steps, pic_tuning *out,
                            void *cuda_stream);

/* Set E^n (N1 doubles: Whitney-1 edge values, line integrals along each edge's tail ->
 * head; PEC entries are forced to 0, Sec. 5.1) and B^{n-1/2} (N2 doubles: Whitney-2 face
 * fluxes) from caller-owned host arrays, copied; either may be NULL to leave it.  Resets
 * the Gauss-law auxiliary flux D = star_eps E (Sec. 3.5.2) and its reference.  Errors: ARG
 * (null handle), CUDA. */
pic_status pic_fields_set(pic_sim *s, const double *E_edges, const double *B_faces_half,
                          void *cuda_stream);

/* Inject n particles of one species: physical positions (z, rho) and momenta u = gamma v
 * in the local (rho, phi, z) frame; charge q and mass m of the physical particle, and the
 * macro-particle weight w.  The ring's source charge is q_src = w q / (2 pi), since the
 * meridian-plane equations are the 3D ones divided by 2 pi.  Each particle is located on
 * the host (the triangle with the largest smallest barycentric coordinate; ties to the
 * lower triangle index), uploaded, and its charge is added to Q^n (Eq. charge).  Only one
 * species per simulation: later calls must repeat q/m and w q.  Errors: ARG (point
 * outside the mesh, species mismatch), OOM (capacity). */
pic_status pic_particles_inject(pic_sim *s, int64_t n, const double *z, const double *rho,
                                const double *u_rho, const double *u_phi, const double *u_z,
                                double q, double m, double weight, void *cuda_stream);

/* Advance n_steps full cycles of Sec. 3 on the stream, each in the order
 *   emission (if set) -> B^{n+1/2} (Eq. full_d_dfl) and the per-triangle field records
 *   -> gather, push (Eqs. DNE, DLE), walk and scatter of J^{n+1/2} (Eq. current) and
 *   Q^{n+1} (Eq. charge) -> E^{n+1} (Eq. full_d_dal, SPAI M) -> re-sort every
 *   sort_interval steps (an implementation step: particles ordered by triangle).
 * Asynchronous: returns once the work is enqueued; the state stays on the device.
 * n_steps = 0 enqueues nothing.  A bounded device wait that gives up (a stalled copy
 * pipeline) is counted on the device and reported as PIC_ERR_TIMEOUT by the next
 * pic_diagnostics, pic_charges_get or pic_charges_get_static.  Errors: ARG (null handle, n_steps < 0), CUDA (a launch or graph
 * call failed). */
pic_status pic_step(pic_sim *s, int64_t n_steps, void *cuda_stream);

/* Synchronous diagnostics (Sec. 3.5, Sec. 5.1.1) and optional field read-back:
 * E_out (N1), B_out (N2, B^{n-1/2}), J_out (N1, J^{n-1/2} of the last step in physical
 * units), each a caller-owned host array or NULL.  out may be NULL too: no reductions
 * run, only the requested arrays are copied (a plain field read-back).  The reductions
 * run on the device.  Errors: ARG (null handle), TIMEOUT (a bounded device wait of an
 * earlier step gave up: the state is invalid), OOM, CUDA. */
pic_status pic_diagnostics(pic_sim *s, pic_diag *out, double *E_out, double *B_out,
                           double *J_out, void *cuda_stream);

/* Node charges in physical units (N0 each, may be NULL): Q^n, Q^{n-1} and the charge
 * absorbed at walls during the last step.  Synchronous.  Errors: ARG, OOM, CUDA, TIMEOUT
 * (a bounded device wait of an earlier step gave up; nothing is written). */
pic_status pic_charges_get(pic_sim *s, double *Q, double *Q_prev, double *Q_absorbed,
                           void *cuda_stream);

/* Same outputs as pic_charges_get, for callers that must not allocate device memory: a
 * process whose device memory is already committed to another allocator's pool (where
 * a new cudaMalloc would fail or fragment it), or a code path that is not allowed to
 * allocate, such as the inside of a time loop with a fixed memory budget.  The paper has
 * no counterpart; this is a library convenience.
 * It calls no cudaMalloc or cudaFree and no allocating library routine.  Its device
 * scratch is a fixed array inside the library (3 x 131072 doubles, 3 MB) that every GPU
 * which loads the library keeps until the process exits.  The first call on a device
 * looks up that array's device address on the current device; make the first call
 * before any stream capture.  Meshes with more than 131072 nodes are rejected with
 * PIC_ERR_ARG (use pic_charges_get).  All calls share the one array, so calls whose GPU
 * work overlaps (different streams or threads) race; each call synchronises its stream
 * before returning.  Q, Q_prev, Q_absorbed: N0 doubles each, or NULL.  TIMEOUT as for
 * pic_charges_get (checked before anything is written). */
pic_status pic_charges_get_static(pic_sim *s, double *Q, double *Q_prev, double *Q_absorbed,
                                  void *cuda_stream);

/* Number of particle slots in use (live and removed-but-not-yet-compacted). */
pic_status pic_particles_count(pic_sim *s, int64_t *n_slots, void *cuda_stream);

/* Particle state, synchronous: for each of the n_slots slots, pid (the 0-based global
 * injection index), tri (-1 for removed particles), lambda (3 doubles) and u (3 doubles).
 * n_cap is the capacity of the output arrays; PIC_ERR_ARG if n_slots > n_cap. */
pic_status pic_particles_get(pic_sim *s, int64_t n_cap, int64_t *pid, int32_t *tri,
                             double *lam, double *u, void *cuda_stream);

/* Raw device state, for host round trips in the storage format: FP32 slots take 24 bytes
 * (int32 tri, int32 lambda_0, int32 lambda_1 at 2^-22, float u_rho, u_phi, u_z), FP64
 * slots 44 bytes (int32 tri, double lambda_0, lambda_1, u_rho, u_phi, u_z), stored as
 * structure-of-arrays with a stride of n_slots rounded up to a multiple of 32 slots: all
 * tri values, then (from byte 4 * stride) all lambda_0, and so on, so that every array
 * starts on a 128-byte boundary of the buffer (host -> device copies from less aligned
 * starts run ~15% slower).  A buffer for n_slots slots holds pic_particles_raw_size bytes
 * (stride x bytes per slot); the padding slots are neither read nor written.
 * pic_particles_raw_get copies the first n_slots slots device -> host (n_slots at most
 * the count from pic_particles_count); pic_particles_raw_set copies n_slots slots host ->
 * device and makes n_slots the slot count (at most the capacity; particle ids are kept).
 * Both are asynchronous on the stream; host buffers should be page-locked. */
pic_status pic_particles_raw_bytes(pic_sim *s, int64_t *bytes_per_particle);
/* Bytes of a raw host buffer of n_slots slots (the layout above).  Errors: ARG (null
 * output, negative count). */
pic_status pic_particles_raw_size(pic_sim *s, int64_t n_slots, int64_t *bytes);
pic_status pic_particles_raw_get(pic_sim *s, void *host_dst, int64_t n_slots,
                                 void *cuda_stream);
pic_status pic_particles_raw_set(pic_sim *s, const void *host_src, int64_t n_slots,
                                 void *cuda_stream);

/* n_steps steps of Sec. 3's cycle for a particle state that lives in page-locked host
 * memory between steps (raw layout above, n_slots slots, n_slots at most the capacity):
 * every step uploads it, steps, and writes it back.  Slots beyond the live count after a
 * re-sort removed particles are unspecified on return.  Uploads and downloads run on
 * internal streams, chunk by chunk: the download of one step overlaps the upload of the
 * next, and (FP32 build, kernel timing off) after the first step the particle kernel runs
 * on each chunk as soon as it has landed and each chunk is written back as soon as it is
 * pushed (after the re-sort, on a re-sort step); the result is bit-identical to stepping
 * on the device.  The call is asynchronous on cuda_stream, which waits for the last
 * download.  Errors: PIC_ERR_ARG
 * (null state, bad counts), PIC_ERR_STATE (an emitter is set: the slot count would grow),
 * PIC_ERR_CUDA.  The host buffer must stay untouched until the stream reaches that point. */
pic_status pic_step_host(pic_sim *s, void *host_state, int64_t n_slots, int64_t n_steps,
                         void *cuda_stream);

/* Device time of the particle kernel over the steps enqueued since the last call
 * (CUDA events around each launch on the step's stream); synchronous.  Writes the
 * total milliseconds and the number of launches. */
pic_status pic_kernel_timing(pic_sim *s, int32_t enable, double *push_ms, int64_t *launches,
                             void *cuda_stream);

/* Number of kernels this library has enqueued for execution in the process so far, on
 * any device and stream (launched directly, or as nodes of a replayed CUDA graph: a graph
 * adds its kernels at each replay, its capture adds none).  Not an operation of the
 * paper; a benchmark reads it before and after a timed region.  Errors: ARG (NULL out). */
pic_status pic_launch_count(int64_t *out);

/* ---- Surrogate network ensemble (not in the paper) ------------------------------------
 * An ensemble of n_members multilayer perceptrons with layer widths sizes[0..n_layers]
 * (inputs first): hidden layers z = x W^T + b followed by the tanh form of GELU, a linear
 * output layer; trained on mean-squared error with Adam.  It stands in for the simulation
 * where the members agree (the caller gates on their spread).  Parameters per member: for
 * each layer W (n_out x n_in, row-major) then b (n_out), members one after another.
 * Device memory comes from the allocator hook, like the simulations'.  max_batch bounds
 * the training batch and the rows of pic_mlp_grad; inference is chunked.  Limits:
 * 1..64 members, 1..16 layers, widths 1..4096, max_batch 1..2^20.  Host arrays are
 * caller-owned and copied; device arrays (X, T, Y) are caller-owned CUDA memory on the
 * network's device.  Errors of every call: ARG (null handle or pointer, a limit above),
 * OOM, CUDA, and TIMEOUT where stated; pic_mlp_destroy releases everything. */
typedef struct pic_mlp pic_mlp;
pic_status pic_mlp_create(int32_t n_members, int32_t n_layers, const int32_t *sizes,
                          int32_t max_batch, pic_mlp **out);
pic_status pic_mlp_param_count(pic_mlp *m, int64_t *per_member);
/* Host copies of all members' parameters (n_members x per_member doubles; stored as FP32).
 * Setting resets the Adam moments.  Synchronous. */
pic_status pic_mlp_params_set(pic_mlp *m, const double *params);
pic_status pic_mlp_params_get(pic_mlp *m, double *params);
/* steps Adam steps (learning rate lr, moments 0.9 / 0.999) on minibatches of `batch` rows
 * drawn with replacement from the n training rows X (device, n x inputs, FP32) and T
 * (device, n x outputs, FP32) by a counter-based hash of (seed, member, step, row): each
 * member sees its own draws.  last_loss (host, n_members, may be NULL) receives each
 * member's loss on its last minibatch; then the call is synchronous. */
pic_status pic_mlp_train(pic_mlp *m, const float *X, const float *T, int64_t n, int32_t batch,
                         int64_t steps, double lr, uint64_t seed, double *last_loss,
                         void *cuda_stream);
/* Gradient of every member's loss over the n <= max_batch rows X, T (device) at the current
 * parameters, to host doubles (n_members x per_member), and the losses (may be NULL).
 * Synchronous.  For checking the backward pass. */
pic_status pic_mlp_grad(pic_mlp *m, const float *X, const float *T, int64_t n, double *grads,
                        double *loss, void *cuda_stream);
/* Outputs Y (device, n_members x n x outputs, FP32) for the rows X (device, n x inputs,
 * FP32).  tensor_cores = 0: FP32 on CUDA cores.  tensor_cores = 1: BF16 operands and FP32
 * accumulation on the tensor cores (tcgen05, every width at most 256; PIC_ERR_ARG
 * otherwise; synchronous, PIC_ERR_TIMEOUT if a bounded wait gave up). */
pic_status pic_mlp_forward(pic_mlp *m, const float *X, float *Y, int64_t n, int32_t tensor_cores,
                           void *cuda_stream);
/* Products of pic_mlp_train and pic_mlp_grad (the forward product and both backward
 * products of every layer) on the tensor cores (tensor_cores != 0: operands rounded to
 * BF16, FP32 accumulation in TMEM) or on CUDA cores in FP32 (0, the default).  Products
 * wider than 256 in N or K stay on CUDA cores.  A bounded tensor-core wait that gives up
 * makes the call that ran it return PIC_ERR_TIMEOUT.  Errors: ARG (a width above 256). */
pic_status pic_mlp_set_training(pic_mlp *m, int32_t tensor_cores);
/* Bound of the tensor-core inference kernel's waits (pic_mlp_forward with tensor_cores):
 * the number of polls, each suspending the waiting thread for at most a system-set time,
 * that a wait for a weight chunk, a product or a tile's operand makes before it gives up.
 * Default 4194304.  A block whose wait gives up stops, waits with the default bound for
 * its own copies and products still in flight, frees its tensor memory and exits; the
 * forward call then returns PIC_ERR_TIMEOUT and its outputs are undefined.  Not an
 * operation of the paper: it lets a caller (a test) make the waits run out, with 0 polls.
 * The training products keep the default bound.  Errors: ARG (negative count). */
pic_status pic_mlp_set_wait_limit(pic_mlp *m, int64_t polls);
void pic_mlp_destroy(pic_mlp *m);

/* Release a simulation (its device memory included) or a mesh; NULL is ignored.  A mesh
 * must outlive the simulations made from it. */
void pic_sim_destroy(pic_sim *s);
void pic_mesh_destroy(pic_mesh *m);
/* Message of the last failing call on this thread (empty if none); valid until the next
 * failing call on the same thread. */
const char *pic_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PIC_H */
