/*
 * qhp.h - C ABI of the B300 (sm_103a) RPMD / adQTB time-step library.
 *
 * Method: Plé et al., "Routine molecular dynamics simulations including nuclear
 * quantum effects: from force fields to machine learning potentials",
 * arXiv 2212.03137.  Equation numbers follow the order of the paper's numbered
 * display equations (Eq. (1) is the partition function of Sec. II.A).
 *
 * Conventions for every entry point
 *   - units: kcal/mol, Angstrom, amu, ps (time steps are given in fs), e, K;
 *   - arrays are C-contiguous; "[n][3]" means n rows of (x, y, z);
 *   - host pointers are read or written synchronously and remain owned by the
 *     caller; "_device" variants take device pointers (e.g. a torch tensor's
 *     data_ptr()) that the library never frees, and work on the system's stream;
 *   - the library owns all device memory of a system and frees it in
 *     qhp_destroy_system;
 *   - every call returns 0 (QHP_OK) or a negative QHP_ERR_* code; the message
 *     of the last failure on the calling thread is qhp_last_error();
 *   - step calls are asynchronous on the system's stream; a fault found on the
 *     device (non-finite state, neighbour-list overflow) is reported by the next
 *     call that synchronises (qhp_sync, the qhp_get_* calls) or by the next step
 *     call.
 */
#ifndef QHP_H
#define QHP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qhp_system_s* qhp_sys;

enum {
    QHP_OK = 0,
    QHP_ERR_ARG = -1,           /* invalid argument or unsupported size */
    QHP_ERR_CUDA = -2,          /* a CUDA runtime call failed */
    QHP_ERR_TIMEOUT = -3,       /* a bounded device wait ran out */
    QHP_ERR_NONFINITE = -4,     /* NaN/Inf found in the state */
    QHP_ERR_LIST_OVERFLOW = -5, /* neighbour list larger than its buffer */
    QHP_ERR_STATE = -6,         /* call out of order (e.g. step before set_beads) */
    QHP_ERR_NOMEM = -7,         /* device allocation failed */
    QHP_ERR_BOUNDS = -8         /* an index read from device data was out of range (bounds-checked
                                   builds only, built with -DQHP_CHECK; plain builds never check) */
};

enum { QHP_FP64 = 0, QHP_MIXED = 1 };
enum { QHP_THERMO_PILE = 0, QHP_THERMO_ADQTB = 1, QHP_THERMO_NVE = 2 };
enum { QHP_ADAPT_NONE = 0, QHP_ADAPT_SIMPLE = 1, QHP_ADAPT_RATIO = 2 };
enum { QHP_INTEGRATOR_BAOAB = 0, QHP_INTEGRATOR_BCOCB = 1 };

/* Interatomic potential V (the paper is independent of V; this is a flexible
 * q-SPC/Fw-style water): O-O Lennard-Jones shifted to 0 at rc, damped-shifted-
 * force Coulomb (damping alpha, 1/A) on all pairs of different molecules,
 * 1/2 k_b (r - r0)^2 per O-H bond and 1/2 k_theta (theta - theta0)^2 per angle.
 * q_H = -q_O / 2.  skin is the Verlet-list buffer (r_list = rc + skin). */
typedef struct {
    double eps, sigma, q_O;
    double k_b, r0, k_theta, theta0; /* theta0 in radians */
    double alpha, rc, skin;
    double m_O, m_H;
} qhp_ff;

/* Thermostat.  PILE (Sec. III.A.1, Eq. (16)): friction gamma0 on the centroid
 * and max(gamma0, omega_n) on mode n > 0.  ADQTB (Sec. II.B, Sec. III.B): single
 * bead, colored noise of power Theta(omega) gamma(omega)/gamma0 per segment of
 * n_seg steps, cut at omega_cut (cm^-1; <= 0 means no cut), gamma(omega)
 * adapted per atom type at every segment end (adapt = QHP_ADAPT_*, rate
 * a_gamma in ps^-1 per kcal/mol, RATIO time tau_ratio_ps) and clamped at
 * gamma_min_frac * gamma0.  NVE: no friction and no noise on any mode (the
 * ring-polymer equations of motion, Eq. (9), integrated as B A A B).
 * integrator: QHP_INTEGRATOR_BAOAB (exact free ring-polymer flow A) or
 * QHP_INTEGRATOR_BCOCB (Sec. III.A.1: A(dt/2) of every internal mode replaced by its
 * Cayley transform, a rotation by 2 atan(omega dt/4) instead of omega dt/2, stable for
 * any omega dt). */
typedef struct {
    int kind;
    double gamma0;        /* ps^-1 */
    double dt_fs;
    int n_seg;
    double omega_cut_cm;
    double a_gamma;
    double gamma_min_frac;
    int adapt;
    double tau_ratio_ps;
    int integrator;
} qhp_thermo;

/* Estimators at the current state (kcal/mol).
 * potential  = U_P = (1/P) sum_i V(x_i)                       (Eq. (3))
 * spring     = sum_{n>0} 1/2 m omega_n^2 Q_n^2                 (Eq. (1))
 * kinetic_nm = sum_n P_n^2 / 2m                               (Eq. (7))
 * kinetic_cv = 3N kT/2 - (1/2P) sum_i (x_i - Q_0).F(x_i)      (Eq. (6))
 * fdt_delta  = adQTB: mean of |Delta_bar_FDT,z(omega_j)| (Eq. (21), the type mean of
 *              Sec. III.B.2, kcal/mol) over both atom types and the n_seg + 1 frequency bins
 *              of the last completed segment, with the gamma that segment ran with; 0 before
 *              the first segment end and without adQTB */
typedef struct {
    double potential, spring, kinetic_nm, kinetic_cv, fdt_delta;
    double bonded, nonbonded, reserved;
} qhp_energy;

typedef struct {
    int n_atoms, P, precision, list_mode; /* list_mode 1: centroid Verlet list, 0: all pairs */
    int64_t step, rebuilds, list_entries, list_capacity;
    int64_t kernel_launches;              /* kernels this system has launched so far */
    int n_cells_per_edge, reserved;
} qhp_info;

/* Create a system of n_atoms atoms in a cubic periodic box of edge box_L (A): the
 * N-atom system whose quantum partition function Eq. (1) of Sec. II.A approximates by
 * P ring-polymer replicas.  type[i]: 0 = O, 1 = H.  Molecules are consecutive
 * (O, H, H) triples with molecule[i] = i / 3.  pos: [n_atoms][3] initial positions
 * (A), used as the centroids Q_0 (the n = 0 mode of Eq. (4)).  precision: QHP_FP64 or
 * QHP_MIXED.  Allocates nothing on the device until qhp_set_beads.  Returns
 * QHP_ERR_ARG for other layouts and for n_atoms >= 2^26.
 * qhp_destroy_system frees the system's device memory, stream and graphs (the handle is
 * invalid afterwards; NULL is accepted).  Neither has a counterpart in the paper: they
 * are the lifetime of the state the paper's equations act on. */
int qhp_create_system(qhp_sys* out, int n_atoms, const int* type, const int* molecule,
                      const double* pos, double box_L, int precision);
int qhp_destroy_system(qhp_sys sys);

/* Set the potential (copied).  The first call must precede qhp_set_beads; rc must be
 * below box_L/2.  Later calls may change eps, sigma, q_O, k_b, r0, k_theta, theta0 and
 * alpha only (QHP_ERR_STATE otherwise); the next step or force call re-evaluates the
 * forces with them. */
int qhp_set_forcefield(qhp_sys sys, const qhp_ff* ff);

/* Allocate the P-bead state and initialise it (Eqs. (4), (7)): Q_0 = input
 * positions, Q_n ~ N(0, kT/(m omega_n^2)) for n > 0, P_n ~ N(0, m kT), drawn
 * from Philox4x32-10 with key = seed.  P must be a power of two, 1 <= P <= 64.
 * Resets the step counter. */
int qhp_set_beads(qhp_sys sys, int P, double temperature_K, uint64_t seed);

/* Set the thermostat and time step (copied).  For ADQTB, P must be 1 and
 * n_seg a power of two in [4, 2048]; the first noise segment is generated here. */
int qhp_set_thermostat(qhp_sys sys, const qhp_thermo* th);

/* Multiple time stepping with ring-polymer contraction (Sec. III.A.2, Eqs. (18)-(20)).
 * V = V_s + V_f with V_f the bonded terms (on all P beads) and V_s the nonbonded ones,
 * evaluated on contracted_beads beads: the Fourier interpolant of the contracted_beads
 * lowest-frequency normal modes at equally spaced imaginary times (0 means P: no
 * contraction).  With n_alt >= 1 each qhp_step_rpmd step is one outer step
 * B_s(n dt/2) [B_f(dt/2) A O A B_f(dt/2)]^n B_s(n dt/2) of n_alt inner steps of the
 * thermostat's dt (the step counter advances by n_alt); n_alt = 0 returns to plain BAOAB.
 * Needs an initialised mixed-precision system with the PILE or NVE thermostat
 * (QHP_ERR_STATE otherwise); contracted_beads must be a power of two dividing P.
 * qhp_get_energy and qhp_get_forces keep their full-ring-polymer definitions. */
int qhp_set_respa(qhp_sys sys, int n_alt, int contracted_beads);

/* Advance n BAOAB steps (Eq. (17)) with the PILE thermostat, or with the adQTB
 * O step for qhp_step_adqtb.  Asynchronous; n >= 0. */
int qhp_step_rpmd(qhp_sys sys, int n);
int qhp_step_adqtb(qhp_sys sys, int n);

/* Evaluate bead forces at the current modes (no time step). */
int qhp_compute_forces(qhp_sys sys);

/* Synchronise the stream and report device-side faults. */
int qhp_sync(qhp_sys sys);

/* Estimators at the current state (the qhp_energy fields above; Eqs. (3), (6), (7),
 * (21)).  Synchronous; out is a host struct. */
int qhp_get_energy(qhp_sys sys, qhp_energy* out);
/* Bead forces F_i = -grad V(x_i) of the last force evaluation (the per-bead gradient of
 * U_P, Eq. (3), before the projection of Eqs. (10)-(11)), out[P][n_atoms][3] host,
 * kcal/mol/A.  Synchronous. */
int qhp_get_forces(qhp_sys sys, double* out);
/* Centroids Q_0 = the n = 0 normal mode (Eq. (4) with T_i0 = 1/sqrt(P), so Q_0 is the
 * bead average), out[n_atoms][3] host, A (unwrapped).  Synchronous. */
int qhp_get_centroid(qhp_sys sys, double* out);
/* Bead positions x_i = sqrt(P) sum_n T_in Q_n in FP64 (Eq. (4)), out[P][n_atoms][3]. */
int qhp_get_beads(qhp_sys sys, double* out);
/* Normal-mode state, Q[n_atoms][3][P] (A) and Pm[n_atoms][3][P] (amu A/ps). */
int qhp_get_modes(qhp_sys sys, double* Q, double* Pm);
/* Replace the mode state (copied); the next step re-evaluates forces and the list. */
int qhp_set_modes(qhp_sys sys, const double* Q, const double* Pm);
/* Device-pointer variants: same layouts, on the system's stream. */
int qhp_set_modes_device(qhp_sys sys, const double* Q, const double* Pm);
int qhp_get_modes_device(qhp_sys sys, double* Q, double* Pm);
int qhp_get_forces_device(qhp_sys sys, double* out);

/* Checkpoint (no counterpart in the paper: a restart facility around the state its
 * equations evolve): opaque blob of the whole dynamical state (modes, forces, step,
 * adQTB gamma, noise segment and records).  qhp_get_state with buf == NULL writes the
 * required size to *size; otherwise buf (host, caller-owned, *size bytes) receives the
 * blob, QHP_ERR_ARG if *size is too small.  qhp_set_state restores a blob taken from a
 * system of the same size, bead count, precision and noise-segment length
 * (QHP_ERR_ARG otherwise); stepping on from it gives the same trajectory bit for bit. */
int qhp_get_state(qhp_sys sys, void* buf, size_t* size);
int qhp_set_state(qhp_sys sys, const void* buf, size_t size);

/* adQTB: gamma_z(omega_j), out[2][n_seg + 1] (type 0 = O, 1 = H), ps^-1. */
int qhp_get_gamma(qhp_sys sys, double* out);
int qhp_set_gamma(qhp_sys sys, const double* in);
/* adQTB: current colored-noise segment u[n_seg][3 n_atoms] (sqrt(kcal/mol)) and
 * the records of the current segment v[n_seg][3n] (A/ps), F[n_seg][3n] (amu A/ps^2). */
int qhp_get_qtb_noise(qhp_sys sys, float* u);
int qhp_get_qtb_records(qhp_sys sys, float* v, float* F);

/* Centroid neighbour structures (Sec. III.A.3), for inspection and tests.
 * qhp_build_list rebuilds them from the current centroids.
 * qhp_get_cells: cell id of each atom [n_atoms] and the sorted order
 * (position -> atom) [n_atoms].  qhp_get_list_pairs: the unordered pairs
 * (i < j, atom indices) of the list, at most cap of them; *count receives the
 * total. */
int qhp_build_list(qhp_sys sys);
int qhp_get_cells(qhp_sys sys, int* cell, int* order);
int qhp_get_list_pairs(qhp_sys sys, int64_t* pairs, int64_t cap, int64_t* count);
/* The list row of one atom: partner atom indices (in list order, at most cap of them);
 * *count receives the row length. */
int qhp_get_list_row(qhp_sys sys, int atom, int* partners, int cap, int* count);

int qhp_get_info(qhp_sys sys, qhp_info* out);

/* Measurement hooks.  With profiling on, every step records CUDA events on the
 * system's stream around its stages (they are captured into the step graph);
 * qhp_get_profile synchronises and returns the stage durations of the last step
 * (ms): B-A-O-A + bead positions, list check/rebuild, nonbonded pair kernel,
 * bonded kernel, force projection + B, and the whole step. */
typedef struct {
    float integrate_ms, list_ms, pair_ms, bonded_ms, project_ms, step_ms;
} qhp_profile;
int qhp_set_profiling(qhp_sys sys, int on);
int qhp_get_profile(qhp_sys sys, qhp_profile* out);
/* Number of bead pairs (each unordered pair once, summed over beads) within rc
 * at the current positions, and how many of them are O-O (LJ) pairs. */
int qhp_count_pairs(qhp_sys sys, int64_t* pairs, int64_t* oo_pairs);
/* Differentiation (the paper has no counterpart; FP64 kernels in either precision).
 * theta = (eps, sigma, q_O, k_b, k_theta) of the current force field, q_H = -q_O/2.
 *
 * qhp_energy_grad: U_P = (1/P) sum_b V(x_b) (Eq. (3), with the DSF self term) at the
 * current bead positions, dU_P/dx = -F_b/P as out[P][n_atoms][3] (host, may be NULL)
 * and dU_P/dtheta[5] (host, may be NULL).  Synchronous.
 * qhp_energy_grad_device: the same with device arrays; if x (device [P][n_atoms][3])
 * is not NULL the bead positions first become the system's modes (momenta kept) and the
 * list is rebuilt around them.  energy and dE_dtheta are host pointers (may be NULL).
 *
 * qhp_segment_grad: J = (1/K) sum_{k=1..K} a(Q_k) along K BAOAB steps (Eq. (17)) from
 * the current state, with the thermostat noise of those steps held fixed, and dJ/dtheta
 * by the adjoint of the FP64 step (Hessian-vector products of the forces, exact).
 * observable 0: the potential energy at the centroid V(Q_0); 1: the mean O-H bond
 * length over beads and both bonds of every molecule.  The forward trajectory is
 * replayed from host checkpoints taken every `block` steps (device memory for block + 1
 * mode arrays).  Needs QHP_FP64 and the PILE or NVE thermostat (QHP_ERR_STATE
 * otherwise); K, block >= 1.  The system is left in the state it had before the call.
 * Synchronous; J and dJ_dtheta[5] are host pointers. */
int qhp_energy_grad(qhp_sys sys, double* energy, double* dE_dx, double* dE_dtheta);
int qhp_energy_grad_device(qhp_sys sys, const double* x, double* energy, double* dE_dx, double* dE_dtheta);
int qhp_segment_grad(qhp_sys sys, int K, int block, int observable, double* J, double* dJ_dtheta);

/* Free-energy differences by path-integral BAR (Sec. V, Perspective 2, Eqs. (27)-(28);
 * the single-bead variant of Appendix A).
 * qhp_state_energies: at the current beads, out[4] = {U_P(A), U_P(B), V_A(x_0), V_B(x_0)}:
 * the bead-averaged potential (Eq. (3)) and the potential of bead 0 alone, for the two
 * parameter sets theta_A, theta_B = (eps, sigma, q_O, k_b, k_theta) (q_H = -q_O/2; the
 * other terms as set by qhp_set_forcefield).  FP64, synchronous.
 * qhp_bar: Dlt F_AB = F_B - F_A (kcal/mol) from dU = U_B - U_A sampled in state A
 * (dU_A[n_A]) and in state B (dU_B[n_B]) (host arrays), beta in (kcal/mol)^-1: the
 * self-consistent solution of Eqs. (27)-(28), iterated from C = ln(n_B/n_A)/beta until C
 * moves by less than tol (QHP_ERR_STATE after 10000 iterations).  Pass bead-averaged
 * differences for PI-BAR or single-bead ones for the single-bead estimator.  The paper's
 * hydration free energies need solute parameters and are not reproduced. */
int qhp_state_energies(qhp_sys sys, const double* theta_A, const double* theta_B, double* out);
int qhp_bar(const double* dU_A, int n_A, const double* dU_B, int n_B, double beta, double tol, double* dF,
            int* iterations);

/* Batched systems (the paper's bead parallelism extended to many independent systems;
 * no counterpart in the paper).  A batch steps n_sys initialised mixed-precision systems
 * with the PILE or NVE thermostat (no RESPA) together: each step is one CUDA graph holding
 * one cooperative launch over every system - integrate (with each system's list check, run
 * by the block that finishes the system), forces (pair items of every bead count, small-box
 * path and warps-per-atom setting and the bonded items, added as int64 fixed point),
 * projection: three phases between grid barriers, persistent blocks over (system, group)
 * work items - plus one conditional node per system that runs only when that system's list
 * check fired: its list rebuild, forces and projection with the single-system kernels.
 * kernels_per_step counts the batched launches (1).  Results are bit-identical to stepping
 * every system alone.  In qhp_batch_info, grid_integrate and grid_project are the launch's
 * blocks, grid_pair its half blocks (pair and bonded items; grid_bonded is 0) and items_pair
 * its pair items; in qhp_batch_get_profile, integrate_ms, pair_ms (pair and bonded) and
 * project_ms are the launch's phases from device clock stamps, list_ms the conditional
 * bodies and bonded_ms 0.
 *
 * A grid barrier that waits longer than the batch's wait limit (default 2 s;
 * qhp_batch_set_wait_limit, 1e3 .. 1e11 ns) gives up: the launch ends and the next
 * qhp_batch_sync returns QHP_ERR_TIMEOUT (the members' state is then undefined).
 * qhp_selftest_grid_barrier runs the barrier with one arrival that never comes, so that
 * every wait runs out after wait_ns (1e3 .. 1e10): it returns QHP_ERR_TIMEOUT with the
 * ST_TIMEOUT bit (4) in *status when the time limit works.  The systems stay owned by the caller and must
 * outlive the batch; while batched, their work runs on the batch's stream (member calls
 * such as qhp_get_modes stay valid and ordered), and qhp_set_stream must not be called
 * on them.  qhp_batch_step is asynchronous; qhp_batch_sync waits and reports the first
 * member fault.
 *
 * qhp_autotune: time the pair kernel of one system with 1, 2 and 4 warps per atom and
 * keep the fastest (*warps_per_atom receives it; forces are recomputed with it).
 * qhp_batch_autotune: the same once per bead count present (on its largest member),
 * applied to every member with that bead count; tuned[7] receives W for P = 1, 2, 4,
 * ..., 64 (0 where absent; may be NULL). */
typedef struct qhp_batch_s* qhp_batch;
typedef struct {
    int n_sys, kernels_per_step;
    int64_t atom_beads, steps, rebuilds, kernel_launches;
    int grid_integrate, grid_pair, grid_bonded, grid_project;
    int items_pair, reserved;
} qhp_batch_info;
int qhp_create_batch(qhp_batch* out, int n_sys, const qhp_sys* systems);
int qhp_destroy_batch(qhp_batch batch);
int qhp_batch_step(qhp_batch batch, int n);
int qhp_batch_sync(qhp_batch batch);
int qhp_batch_set_stream(qhp_batch batch, void* stream);
int qhp_batch_autotune(qhp_batch batch, int reps, int* tuned);
int qhp_batch_get_info(qhp_batch batch, qhp_batch_info* out);
int qhp_batch_set_wait_limit(qhp_batch batch, long long wait_ns);
int qhp_selftest_grid_barrier(long long wait_ns, unsigned* status);
/* Stage durations of the last batched step (ms), as qhp_get_profile: integrate (with the
 * list checks), conditional bodies, forces, projection.  Synchronises the batch's stream. */
int qhp_batch_get_profile(qhp_batch batch, qhp_profile* out);
int qhp_autotune(qhp_sys sys, int reps, int* warps_per_atom);
/* Fix the warps per atom of the mixed pair kernel (1, 2 or 4; 0 = the default for P:
 * 4 if P >= 16, else 1).  The forces do not depend on it: every row is summed in FP32 over
 * fixed blocks of 32 list entries, each block sum is converted to int64 fixed point once,
 * and the integers are added, so every setting gives the same bits.
 *
 * qhp_set_pair_skip: the mixed pair kernel walks each list row in (partner type, distance)
 * order and stops a row's group at the first block of entries whose anchor distance exceeds
 * rc + 2 max|x_ib - A_i| (the largest bead offset from its anchor since the list build):
 * no bead pair there can come within rc (Sec. III.A.3 lists pairs by centroid, so the list
 * holds pairs up to rc + skin).  enabled = 0 evaluates every entry instead; the results are
 * the same bits either way (a verification and measurement hook).  Default 1. */
int qhp_set_pair_warps(qhp_sys sys, int warps_per_atom);
int qhp_set_pair_skip(qhp_sys sys, int enabled);

/* Launch mode of qhp_step_rpmd / qhp_step_adqtb.  use_graphs = 1 (default): each
 * step replays one captured CUDA graph whose list-rebuild chain sits behind a
 * conditional node.  use_graphs = 0: the same kernels are launched one by one and
 * the rebuild chain is launched every step, its kernels returning at once when no
 * rebuild is due (for kernel-by-kernel profilers, which do not see kernels inside
 * conditional graph bodies).  Results are bit-identical in both modes. */
int qhp_set_graph_mode(qhp_sys sys, int use_graphs);
/* Use an external CUDA stream (cudaStream_t passed as void*); NULL restores the
 * library's own stream. */
int qhp_set_stream(qhp_sys sys, void* stream);

/* The spring, normal-mode kinetic and centroid-virial kinetic estimators of
 * qhp_get_energy, computed on caller-owned device arrays without allocating any
 * device memory.  The paper has no counterpart: this is a library convenience for
 * callers that cannot allocate at the point of use (inside another framework's
 * CUDA-graph capture, where cudaMalloc is not allowed; on threads that must not
 * synchronise with the device; under an application-wide memory pool).
 *   Q, Pm : device [n_atoms][3][P] modes (A) and momenta (amu A/ps), as qhp_get_modes_device;
 *   F     : device [P][n_atoms][3] bead forces (kcal/mol/A), as qhp_get_forces_device,
 *           or NULL (the virial term is then 0);
 *   mass  : device [n_atoms] (amu);  out: device [3] = spring, kinetic_nm, kinetic_cv (kcal/mol);
 *   stream: cudaStream_t (as void*), NULL for the legacy default stream.
 * Work is enqueued asynchronously on the stream.  Partial sums live in one fixed
 * device array of the library (1.5 MiB per GPU, held until the process exits):
 * n_atoms may be at most 65536 * (64 / P), larger inputs return QHP_ERR_ARG.  Every
 * call made outside a stream capture looks up that array's address on the current device
 * (cudaGetSymbolAddress), so a device reset between calls is harmless; a call inside a
 * capture reuses the address of the last such call, so make one call on each device
 * before any stream capture (QHP_ERR_STATE otherwise), and do not replay a captured graph
 * across a device reset.  Every call reuses the same array, overwriting
 * it entirely (nothing needs clearing); calls that overlap on the GPU, e.g. on two
 * streams at once, race on it and must be serialised by the caller.  P must be a
 * power of two in [1, 64]. */
int qhp_estimators_noalloc(int n_atoms, int P, double temperature, const double* Q, const double* Pm,
                           const double* F, const double* mass, double* out, void* stream);

/* Message of the last failure on this thread ("" if none).  Thread-local rather than
 * per system: failures of qhp_create_system or qhp_bar have no system to attach to.
 * The pointer stays valid until the next failing call on the same thread. */
const char* qhp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
