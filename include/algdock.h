/*
 * algdock.h - C ABI of the GB300 (sm_103a) library for the hot path of AlGDock's binding potential
 * of mean force (BPMF) method: Hamiltonian Monte Carlo of a flexible ligand against a rigid
 * receptor represented by interpolation grids, over many thermodynamic states at once, with
 * Hamiltonian replica exchange, reduced-energy (u_kn) evaluation and MBAR.
 * Paper: D. D. L. Minh, "Alchemical Grid Dock (AlGDock): Binding Free Energy Calculations between
 * Flexible Ligands and Rigid Receptors", arXiv:1507.03703.
 *
 * Call groups, in the order below: lifecycle (with the method's adjustable arguments); grids; the
 * all-FP64 evaluation path and the gather probe; ligand and states; sampling (HMC trial,
 * external-coordinate moves, forces and energies, replica exchange, one whole cycle); the
 * context's own run (replicas held by the context); estimation (u_kn, MBAR, equilibration
 * detection); protocol initialization;
 * multi-ligand batches; the end points (target force field and free energy perturbation); the
 * learned pose proposal; checkpoint and resume; the allocation-free MBAR.
 *
 * Conventions for every call:
 *  - Units: A, kcal/mol, amu, fs, K, elementary charge.
 *  - Every call returns algdock_status (ALGDOCK_OK = 0).  No C++ exception crosses the ABI.
 *    On failure algdock_last_error(ctx) returns a message owned by the context, valid until the
 *    next call on that context.
 *  - Array arguments are owned by the caller.  Unless stated otherwise they must be DEVICE
 *    pointers on the context's device (e.g. torch CUDA tensors' data_ptr()); arguments marked
 *    "host or device" are detected with cudaPointerGetAttributes.  Arrays are C-contiguous.
 *  - Work is enqueued on the stream set by algdock_set_stream (default: the legacy stream) and is
 *    asynchronous unless a call returns host scalars (then it synchronises that stream).
 *  - The context copies grids, ligand and state tables into device memory it owns.
 *  - A context is not thread-safe; use one per host thread.
 */
#ifndef ALGDOCK_H
#define ALGDOCK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ALGDOCK_OK = 0,
  ALGDOCK_E_INVALID = 1,       /* bad argument: null pointer, size, shape, missing setup */
  ALGDOCK_E_CUDA = 2,          /* a CUDA runtime call failed */
  ALGDOCK_E_OOM = 3,           /* device allocation failed */
  ALGDOCK_E_NUMERIC = 4,       /* non-finite input where a finite one is required */
  ALGDOCK_E_NOT_CONVERGED = 5, /* MBAR reached max_iter */
  ALGDOCK_E_STATE = 6          /* call order: grids, ligand or states not loaded */
} algdock_status;

typedef struct algdock_ctx algdock_ctx;

/* A regular lattice: node (i, j, k) at origin + spacing * (i, j, k); arrays are [nz][ny][nx]
 * (x fastest).  Each n >= 2. */
typedef struct {
  double origin[3];
  double spacing;
  int32_t n[3];
} algdock_grid_desc;

/* Ligand topology and parameters (host pointers; copied by algdock_ligand_load).
 * Sampling force field ("Thermodynamic Cycle"; GAFF-like):
 *   bonds     k (r - r0)^2;   angles  k (theta - theta0)^2 (theta0 in rad);
 *   torsions  sum_{n=1..3} V_n/2 (1 + cos(n phi - gamma_n)), V and gamma [n_torsions][3];
 *   nonbonded pairs more than two bonds apart, no cutoff: eps_ij [(R_ij/r)^12 - 2 (R_ij/r)^6]
 *     + 332.0637 q_i q_j / r with eps_ij = sqrt(eps_i eps_j), R_ij = R*_i + R*_j; pairs exactly
 *     three bonds apart (1-4) scaled by 1/2 (LJ) and 1/1.2 (Coulomb).
 * Receptor-ligand grid factors per atom: sqrt(A_i) = sqrt(eps_i) (2 R*_i)^6 for the repulsive
 * grid, sqrt(B_i) = sqrt(2 eps_i) (2 R*_i)^3 for the attractive grid, q_i for the electrostatic.
 * Index arrays are 0-based int32: bonds [n][2], angles [n][3] (centre in the middle),
 * torsions [n][4].  1 <= n_atoms <= 96. */
typedef struct {
  int32_t n_atoms;
  const double* mass;
  const double* charge;
  const double* rstar;
  const double* eps;
  int32_t n_bonds;
  const int32_t* bonds;
  const double* bond_k;
  const double* bond_r0;
  int32_t n_angles;
  const int32_t* angles;
  const double* angle_k;
  const double* angle_theta0;
  int32_t n_torsions;
  const int32_t* torsions;
  const double* torsion_V;
  const double* torsion_gamma;
} algdock_ligand;

/* Flat-bottom harmonic restraint on the ligand centre of mass, Eq. (binding_site):
 * U_I = 0 if d <= d0, else k/2 (d - d0)^2, d = |COM - site|.  The paper's k = 10000 kJ/(mol nm^2)
 * is 23.9006 kcal/(mol A^2); d0 = 6 A. */
typedef struct {
  double site[3];
  double k;
  double d0;
} algdock_restraint;

/* Counters written by algdock_hmc_cycle (added to, not overwritten). */
enum {
  ALGDOCK_CNT_ACCEPTED = 0,  /* HMC trials accepted */
  ALGDOCK_CNT_NONFINITE = 1, /* trials whose total energy change was not finite (rejected) */
  ALGDOCK_CNT_OUTSIDE = 2,   /* atom evaluations clamped to the lattice boundary */
  ALGDOCK_N_COUNTERS = 4
};

/* The method's adjustable arguments ("Sampling", "Equilibration and production", "Estimation").
 * They are the settings of the context's own run (algdock_replicas_init, algdock_run) and the
 * defaults that algdock_mbar takes for tol = 0, max_iter = 0 and precision_mode = -1; every other
 * call that takes one of these quantities as an argument uses its argument.
 * algdock_params_default writes: 50 velocity-Verlet steps per HMC trial, 25 exchange sweeps of
 * separations 1..5 per cycle, no external-coordinate moves (the paper's setting is n_external = 20
 * at alpha_max = 0.01 with sigma_ext = 0.6 A), MBAR to 1e-10 kT in at most 10000 iterations in
 * FP64 (precision mode 0), checks off. */
typedef struct {
  int32_t n_steps;        /* velocity-Verlet steps per HMC trial, >= 0 */
  int32_t n_sweeps;       /* exchange sweeps per cycle, >= 0 */
  int32_t max_sep;        /* largest state separation of an exchange attempt, >= 1; n_sweeps * max_sep < 65536 */
  int32_t n_external;     /* external-coordinate moves per replica after each HMC trial, >= 0 */
  double alpha_max;       /* ... at the states with alpha < alpha_max */
  double sigma_ext;       /* translation standard deviation of an external move (A), finite, >= 0 */
  double mbar_tol;        /* > 0 */
  int32_t mbar_max_iter;  /* >= 1 */
  int32_t mbar_precision; /* algdock_mbar's precision_mode, 0..2 */
  /* nonzero: every cycle of algdock_cycle and algdock_run (and algdock_replicas_init) checks its
   * results on the device - positions and energy components finite (else ALGDOCK_E_NUMERIC),
   * every state index inside the table and every ladder's config_of a permutation that agrees
   * with state_of (else ALGDOCK_E_STATE) - and then synchronises the stream.  The arrays keep the
   * cycle's results either way. */
  int32_t checks;
} algdock_params;

/* ---------------------------------------------------------------- lifecycle */
/* Writes the defaults above into *params. */
algdock_status algdock_params_default(algdock_params* params);
/* Creates a context on CUDA device `device`.  seed keys every Philox stream of the context's own
 * run (the calls that take a seed argument use theirs); params may be NULL (the defaults).
 * ALGDOCK_E_INVALID for out-of-range params, ALGDOCK_E_CUDA for a bad device. */
algdock_status algdock_create(int device, uint64_t seed, const algdock_params* params, algdock_ctx** out);
void algdock_destroy(algdock_ctx* ctx);
/* Replaces the context's params (validated as in algdock_create); the next cycle uses them. */
algdock_status algdock_set_params(algdock_ctx* ctx, const algdock_params* params);
/* Reads the context's params and seed (either pointer may be NULL). */
algdock_status algdock_get_params(algdock_ctx* ctx, algdock_params* params, uint64_t* seed);
/* stream: a cudaStream_t (NULL = legacy default stream). */
algdock_status algdock_set_stream(algdock_ctx* ctx, void* stream);
const char* algdock_last_error(const algdock_ctx* ctx);

/* ---------------------------------------------------------------- grids */
/* Raw receptor grids by direct summation over receptor atoms j at every node p (the paper solves
 * the electrostatic grid with APBS; here a direct Coulomb sum with a distance-dependent
 * dielectric 4r stands in for it) - "Thermodynamic Cycle", electrostatic and van der Waals grids:
 *   LJr(p)  = sum_j sqrt(A_j) / r^12          (r >= 0.01 A)
 *   LJa(p)  = -sum_j sqrt(B_j) / r^6          (r >= 2 A)
 *   elec(p) = 332.0637 sum_j q_j / (4 r^2)    (r >= 2 A)
 * Receptor arrays (host or device, double): xyz [n_rec][3], rstar, eps, q [n_rec].
 * Outputs ljr, lja, elec: device float [nz][ny][nx].  Terms in FP32, sums in FP64. */
algdock_status algdock_grids_build(algdock_ctx* ctx, const algdock_grid_desc* desc, int32_t n_rec,
                                   const double* rec_xyz, const double* rec_rstar, const double* rec_eps,
                                   const double* rec_q, float* ljr, float* lja, float* elec);

/* Soft electrostatic cap for a ligand ("Thermodynamic Cycle", soft grids):
 * v_e = vmax_r * min over charged atoms of sqrt(A_i)/|q_i|, so that every atom's electrostatic
 * energy on the soft grid is bounded by its soft repulsive cap.  +inf if no atom is charged.
 * Host-only arithmetic; needs no context. */
algdock_status algdock_soft_elec_cap(const algdock_ligand* lig, double vmax_r, double* vmax_e);

/* Load raw grids (host or device float [nz][ny][nx], energies per unit scale factor) and derive
 * the interpolated lattices ("Thermodynamic Cycle"): the repulsive grid stored as its 4th root
 * (values capped at 1e10 first), the attractive and electrostatic grids as given, and the soft
 * grids vmax_r tanh(LJr/vmax_r) (stored as its 4th root) and vmax_e tanh(elec/vmax_e).  The
 * paper's vmax_r is 10 kJ/mol = 2.3901 kcal/mol per unit factor; vmax_e from
 * algdock_soft_elec_cap (infinite = no cap).  The derivation runs in FP64; lattices are FP32. */
algdock_status algdock_grids_load(algdock_ctx* ctx, const algdock_grid_desc* desc, const float* ljr,
                                  const float* lja, const float* elec, double vmax_r, double vmax_e);

/* ---------------------------------------------------------------- the all-FP64 path
 * The FP64 arm of the precision study (no counterpart in the paper): the same energy function
 * as algdock_energy_force with every operation in FP64, on FP64 lattices and the ligand's FP64
 * parameters (kept by algdock_ligand_load).  One thread per configuration; a study tool, not a
 * fast path. */

/* FP64 lattices from raw grids (host or device double [nz][ny][nx]), derived as algdock_grids_load
 * does (4th root of the capped repulsive grid, tanh-capped soft grids) but kept in FP64.  They
 * are separate from the FP32 lattices. */
algdock_status algdock_grids_load_f64(algdock_ctx* ctx, const algdock_grid_desc* desc, const double* ljr,
                                      const double* lja, const double* elec, double vmax_r, double vmax_e);

/* Components {U_L, U_I, Psi_sg, Psi_g} (comps [N][4] double) and, with force != NULL, the force
 * [N][n_atoms][3] double of the state state_of[n] (NULL: grid weights zero) for configurations
 * x [N][n_atoms][3] float, all in FP64.  Device arrays. */
algdock_status algdock_energy_force_f64(algdock_ctx* ctx, int64_t N, const int32_t* state_of, const float* x,
                                        double* force, double* comps);

/* Measurement aid for the gather roofline (no counterpart in the paper, not a step of the
 * method): n_cells 8-corner gathers from the loaded lattices at cells drawn uniformly (hard float4
 * corners; with soft != 0 also the soft corners), through the lattice records and loads of one
 * atom's trilinear interpolation.  Useful bytes: 96 per cell (three grids; the records' fourth
 * lane is padding), plus 64 with soft.  Time it with events on
 * the context's stream.  sink: a device float that is written only if the folded sum takes an
 * impossible value (it keeps every load live). */
algdock_status algdock_gather_probe(algdock_ctx* ctx, int64_t n_cells, int32_t soft, uint64_t seed, float* sink);

/* ---------------------------------------------------------------- ligand and states */
algdock_status algdock_ligand_load(algdock_ctx* ctx, const algdock_ligand* lig, const algdock_restraint* rest);

/* The shared-memory layout of the bonded forces that algdock_ligand_load and algdock_batch_load
 * build for this ligand's topology (host only: no context, no device).  In each force evaluation
 * the bonded terms run one per lane in rounds of 32, kind by kind (bonds, angles, torsions); the
 * term at position p of kind k writes its role-r force to slot base_k + r n_k + p (base 0,
 * 2 n_bonds, 2 n_bonds + 3 n_angles; n_k the kind's count).  The slots, listed atom by atom, are
 * added by the 32 lanes in runs of Lr = max(ceil(n_slots / 32), ceil(m / 3)) entries (m the
 * largest number of slots of one atom), each lane's partial sum of an atom stored at that atom's
 * last entry in the run.  The term order, the order of the slots within each atom and the lane of
 * each run are chosen against shared-memory bank conflicts.  Outputs (each may be NULL):
 *   term_order [n_bonds + n_angles + n_torsions]: the input term at each position, bonds first;
 *   slots [n_slots = 2 n_bonds + 3 n_angles + 4 n_torsions]: the slot list, atom by atom;
 *   lane_run [32]: the run each lane adds;
 *   wavefronts [2]: the shared-memory wavefronts per force evaluation of the three loads the
 *   layout arranges (each term round's loads of one role's atom positions, the gather's slot
 *   loads at each run position, the owners' loads of each atom's k-th partial sum), counted per
 *   quarter-warp as the largest number of distinct 16-byte addresses (slot or atom) in one of the
 *   8 bank groups (address mod 8): [0] for the input order, [1] for the layout.
 * Deterministic for a topology.  ALGDOCK_E_INVALID for a topology algdock_ligand_load rejects
 * (an index out of range, too many terms, an atom whose slots would meet more than 4 runs). */
algdock_status algdock_gather_layout(const algdock_ligand* lig, int32_t* term_order, uint16_t* slots,
                                     int32_t* lane_run, int32_t* wavefronts);

/* K thermodynamic states (host arrays): temperature T (K), alchemical progress alpha, and the
 * velocity-Verlet time step dt (fs).  Eq. (protocol): the grid weights are
 *   alpha_sg = 1 - (2 alpha - 1)^2,  alpha_g = (2 alpha - 1)^2 / (1 + exp(-1000 (alpha - 1/2))),
 * and u_k(x) = (U_L + U_I + alpha_sg Psi_sg + alpha_g Psi_g) / (k_B T_k).  alpha = NaN marks a
 * state without receptor grids (the warming leg B -> C). */
algdock_status algdock_states_set(algdock_ctx* ctx, int32_t K, const double* T, const double* alpha,
                                  const double* dt_fs);

/* ---------------------------------------------------------------- sampling */
/* One HMC trial for each of n_rep replicas ("Sampling": HMC with n_steps of velocity Verlet and
 * the Metropolis criterion on H = kinetic + U_k).  Replica r is at state state_of[r] (int32,
 * index into the state table).  Momenta are drawn from N(0, k_B T / m) with Philox4x32-10 keyed
 * by seed, counter {atom, rep_offset + r, cycle, 1}; the acceptance uniform from counter
 * {0, rep_offset + r, cycle, 2}.  Energies are FP32 per term and summed in FP64; the energy
 * change and the accept test are FP64.
 *   x        [n_rep][n_atoms][3] float, in/out: the new configuration, or the old one if rejected
 *   comps    [n_rep][4] double out: {U_L, U_I, Psi_sg, Psi_g} of the returned configuration
 *   dH       [n_rep] double out (may be NULL): total energy change of the trial (kcal/mol)
 *   accepted [n_rep] uint8 out (may be NULL)
 *   counters [ALGDOCK_N_COUNTERS] int64 (may be NULL): accumulated, see ALGDOCK_CNT_*  */
algdock_status algdock_hmc_cycle(algdock_ctx* ctx, int64_t n_rep, const int32_t* state_of, float* x,
                                 double* comps, double* dH, uint8_t* accepted, int32_t n_steps, uint64_t seed,
                                 uint64_t cycle, int64_t rep_offset, int64_t* counters);

/* External-coordinate moves ("Sampling"): for each replica r whose state k = state_of[r] has
 * alpha_k < alpha_max (the warming leg's alpha = NaN never qualifies), n_moves moves, each a
 * uniformly random rotation about the centre of mass (the unit quaternion of three uniforms,
 * Shoemake's construction) and a Gaussian translation of sigma (A) per dimension, accepted by the
 * Metropolis criterion u < exp(-(U_k(x') - U_k(x)) / (k_B T_k)).  The paper: alpha_max = 0.01,
 * sigma = 0.6 A, 20 moves after each HMC move.  A rigid move leaves U_L unchanged: comps[r][0] is
 * carried over and U_I, Psi_sg, Psi_g are re-evaluated (FP32 terms, FP64 sums and decision).
 * Philox4x32-10 keyed by seed, counter {d, rep_offset + r, cycle * n_moves + move, 5}: d = 0 the
 * quaternion's 23-bit uniforms, d = 1 the translation (Box-Muller), d = 2 the accept uniform.
 *   state_of [n_rep] int32, x [n_rep][n_atoms][3] float (in/out), comps [n_rep][4] double (in/out:
 *            the components of x on entry, of the returned configuration on exit), all device
 *   accepted [n_rep] int32 (device, may be NULL): incremented by the number of accepted moves
 *   counters [ALGDOCK_N_COUNTERS] int64 (device, may be NULL): accumulated
 * Errors: E_INVALID (negative sizes, sigma < 0 or not finite, non-device pointers), E_STATE (no
 * grids, ligand or states). */
algdock_status algdock_external_moves(algdock_ctx* ctx, int64_t n_rep, const int32_t* state_of, float* x,
                                      double* comps, int32_t n_moves, double alpha_max, double sigma, uint64_t seed,
                                      uint64_t cycle, int64_t rep_offset, int32_t* accepted, int64_t* counters);

/* Energy and force of N configurations, each at its state ("Thermodynamic Cycle": grid
 * interaction energy and sampling force field; Eq. (binding_site); Eq. (protocol) weights), with
 * the arithmetic of one velocity-Verlet force evaluation inside algdock_hmc_cycle.
 *   state_of [N] int32, x [N][n_atoms][3] float (device)
 *   force    [N][n_atoms][3] float out: -dU_k/dx, U_k = U_L + U_I + alpha_sg Psi_sg + alpha_g Psi_g
 *   comps    [N][4] double out (may be NULL): {U_L, U_I, Psi_sg, Psi_g} */
algdock_status algdock_energy_force(algdock_ctx* ctx, int64_t N, const int32_t* state_of, const float* x,
                                    float* force, double* comps);

/* Hamiltonian replica exchange ("Sampling", Eq. (repXacc)) on n_ladders independent ladders of K
 * consecutive states [state_offset, state_offset + K).  config_of [n_ladders][K] int32 (in/out):
 * the slot (0..K-1) holding the configuration at each state; comps [n_ladders][K][4] double: the
 * components of each slot; state_of [n_ladders][K] int32 (out, may be NULL): the new state of each
 * slot, state_offset + k, in the form algdock_hmc_cycle reads.  One sweep attempts, for s = 1..min(max_sep, K-1) and colour 0 then 1,
 * every pair (a, a+s) with floor(a/s) % 2 == colour, accepting if
 * u < exp(-[u_a(y) + u_b(x) - u_a(x) - u_b(y)]) in FP64, u from Philox counter
 * {(sweep*max_sep + s-1)*65536 + a, ladder_offset + l, cycle, 3}.  Requires K <= 1024 and
 * n_sweeps*max_sep < 65536.  attempts / accepts [max_sep][K] int64 (may be NULL) are added to. */
algdock_status algdock_exchange(algdock_ctx* ctx, int32_t n_ladders, int32_t K, int32_t state_offset,
                                const double* comps, int32_t* config_of, int32_t* state_of, int32_t n_sweeps,
                                int32_t max_sep, uint64_t seed, uint64_t cycle, int64_t ladder_offset,
                                int64_t* attempts, int64_t* accepts);

/* One iteration of the paper's loop over a whole run ("Equilibration and production"):
 * an HMC trial of every replica at its state (as algdock_hmc_cycle), the external-coordinate moves
 * if desc->n_external > 0 (as algdock_external_moves), then n_sweeps exchange sweeps on every
 * ladder of every leg (as algdock_exchange), and, if u_kn is given, the snapshot: the reduced
 * energies of every configuration at every state of its leg, formed from the components that the
 * trial's final energy evaluation and the moves left in comps (as algdock_reduced_energies from
 * comps; U_k is linear in the components, so nothing is evaluated twice).  Replicas are leg-major: leg l's chain c holds slots
 * base_l + c K_l + i, base_l = n_chains sum_{m<l} K_m, with config_of laid out the same way
 * ([n_chains][K_l] per leg).  Leg l's ladders are numbered ladder_offset + l n_chains.
 *   x [R][n_atoms][3] float, comps [R][4] double, state_of [R] int32, config_of [R] int32: each host
 *   or device (cudaPointerGetAttributes), read and written; counters [ALGDOCK_N_COUNTERS] int64
 *   (may be NULL) host or device, added to; u_kn (may be NULL) host or device out, leg after leg
 *   [K_l][n_chains K_l] double.
 * On a device that reaches host memory over a coherent link (NVLink-C2C: the device attribute
 * cudaDevAttrHostNativeAtomicSupported), x, comps, state_of, config_of and u_kn in pinned host
 * memory (cudaMemoryTypeHost) are read and written in place by the cycle's kernels.  Other host
 * arrays (pageable ones, and the counters) are copied into device memory the context owns, and
 * back after the cycle.  With any host array
 * the call then synchronises; with device arrays only it is asynchronous like the other calls. */
#define ALGDOCK_MAX_LEGS 8
typedef struct {
  int32_t n_legs;
  int32_t K[ALGDOCK_MAX_LEGS];            /* states per leg */
  int32_t state_offset[ALGDOCK_MAX_LEGS]; /* each leg's first state in the context's table */
  int32_t n_chains;
  int32_t n_steps;                        /* velocity-Verlet steps per HMC trial */
  int32_t n_sweeps, max_sep;              /* exchange sweeps per cycle and largest separation */
  uint64_t seed;
  int64_t rep_offset, ladder_offset;      /* global index of the first replica and ladder */
  int32_t n_external;                     /* external-coordinate moves after the HMC trial (0: none), */
  double alpha_max, sigma_ext;            /* as algdock_external_moves, between the trial and the sweeps */
} algdock_run_desc;
algdock_status algdock_cycle(algdock_ctx* ctx, const algdock_run_desc* desc, uint64_t cycle, float* x, double* comps,
                             int32_t* state_of, int32_t* config_of, int64_t* counters, double* u_kn);

/* ---------------------------------------------------------------- the context's own run */
/* Replicas owned by the context, in algdock_cycle's layout: n_legs legs, leg l with K[l] states
 * starting at state_offset[l] of the state table, n_chains chains per leg; R = n_chains sum K[l]
 * replicas, leg-major, chain c of leg l at slots base_l + c K[l] + i (i = 0..K[l]-1).
 *   x0 [R][n_atoms][3] float, host or device: the starting configurations.
 * Each slot starts at its own state (state_of = state_offset[l] + i, config_of = i), its energy
 * components are evaluated, the counters are zeroed.  rep_offset and ladder_offset are the global
 * indices of the first replica and ladder, as in algdock_run_desc (0 for a one-process run).
 * Replaces any replicas the context held.  Synchronises the stream. */
algdock_status algdock_replicas_init(algdock_ctx* ctx, int32_t n_legs, const int32_t* K, const int32_t* state_offset,
                                     int32_t n_chains, int64_t rep_offset, int64_t ladder_offset, const float* x0);
/* n_cycles cycles of the paper's loop over the context's replicas (algdock_cycle with the
 * context's params and seed), cycles first_cycle .. first_cycle + n_cycles - 1.  u_kn (may be NULL,
 * host or device) receives each cycle's snapshot, cycle after cycle, each laid out as
 * algdock_cycle's u_kn. */
algdock_status algdock_run(algdock_ctx* ctx, int32_t n_cycles, uint64_t first_cycle, double* u_kn);
/* Copies the replicas out (each pointer may be NULL; host or device): x [R][n_atoms][3] float,
 * comps [R][4] double, state_of [R] int32, config_of [R] int32, counters [ALGDOCK_N_COUNTERS]
 * int64.  Synchronises the stream. */
algdock_status algdock_replicas_get(algdock_ctx* ctx, float* x, double* comps, int32_t* state_of,
                                    int32_t* config_of, int64_t* counters);
/* Saves the replicas, their layout, the seed and next_cycle as a checkpoint (the format of
 * algdock_checkpoint_save, arrays "replicas.*"); algdock_replicas_load restores all of them (the
 * grids and ligand must be loaded; the state table comes from the file), so that algdock_run from
 * the restored next_cycle repeats the uninterrupted run bit for bit. */
algdock_status algdock_replicas_save(algdock_ctx* ctx, const char* path, uint64_t next_cycle);
algdock_status algdock_replicas_load(algdock_ctx* ctx, const char* path, uint64_t* next_cycle);

/* ---------------------------------------------------------------- estimation */
/* Reduced energies for MBAR ("Estimation").  If x ([N][n_atoms][3] float) is given, the energy
 * path evaluates each configuration's components into comps ([N][4] double, may then be NULL);
 * if x is NULL, comps is read.  If u_kn is given it receives, for the k_count states starting at
 * k_begin, u_kn[k][n] = (((U_L + U_I) + alpha_sg Psi_sg) + alpha_g Psi_g) / (k_B T_k) in FP64
 * ([k_count][N] double). */
algdock_status algdock_reduced_energies(algdock_ctx* ctx, int64_t N, const float* x, double* comps,
                                        int32_t k_begin, int32_t k_count, double* u_kn);

/* MBAR (Shirts & Chodera 2008, cited in "Estimation") by self-consistent iteration in log-sum-exp
 * form from f = 0, with gauge f_0 = 0:
 *   f_i <- -ln sum_n exp(-u_in) / sum_k N_k exp(f_k - u_kn)
 * until max_i |change| < tol or max_iter iterations.  u_kn [K][N] double (device), N_k [K] int64
 * (host).  precision_mode 0: FP64 throughout; 1: exponentials in FP32 of FP64 arguments, sums in
 * FP64; 2: each sample's column shifted by its minimum (FP64, exact in the result) and stored as
 * FP32, then FP32 arguments, exponentials and Kahan-compensated sums, FP64 only where partial sums
 * meet (K <= 16384; extra scratch K*N*4 bytes).  K <= 65535 in every mode.  tol = 0, max_iter = 0
 * and precision_mode = -1 take the context's params (mbar_tol, mbar_max_iter, mbar_precision).
 * f_k [K] (host) and iters (host) receive the result.  Synchronises.  Returns
 * ALGDOCK_E_NOT_CONVERGED (with the last iterate in f_k) if max_iter is reached. */
algdock_status algdock_mbar(algdock_ctx* ctx, int32_t K, int64_t N, const double* u_kn, const int64_t* N_k,
                            double tol, int32_t max_iter, int32_t precision_mode, double* f_k, int32_t* iters);


/* Automated equilibration detection ("Equilibration and production": statistical inefficiency;
 * the method of Chodera 2016).  For each of S series of length T (series s at a[t * S + s], a
 * device double array, time-major as a history of per-chain values) and each candidate start
 * t0 = c * stride (c < n_cand), the statistical inefficiency of the tail a[t0:],
 *   g = 1 + 2 sum_{t >= 1} (1 - t/N) C(t), C(t) = sum_i (a_i - mu)(a_{i+t} - mu) / ((N - t) var),
 * summed until C(t) first drops to <= 0 (N = T - t0; mu, var of the tail), goes to g [S][n_cand]
 * (device double).  Per series, the t0 that maximises N_eff = N / g (the earliest on ties) goes
 * to t0_best [S] (device int64, may be NULL) and that N_eff to neff_best [S] (device double, may
 * be NULL).  Mean and variance are FP64, the lag products FP32 with FP64 sums across lanes.
 * Errors: E_INVALID unless 2 <= T <= 50000, 1 <= S <= 65535, stride >= 1, n_cand >= 1 and
 * (n_cand - 1) * stride <= T - 2, or for non-device pointers. */
algdock_status algdock_detect_equilibration(algdock_ctx* ctx, int64_t T, int64_t S, const double* series,
                                            int64_t stride, int32_t n_cand, double* g, int64_t* t0_best,
                                            double* neff_best);

/* ---------------------------------------------------------------- protocol initialization
 * "Initialization": a protocol is built state by state.  Parameters of the next state are one
 * thermodynamic-length step away, Delta lambda = s / sigma_0[d l / d lambda], with the standard
 * deviations of the current state's samples.  Seeds for the next state are resampled with weights
 * exp(u_k(x_i) - u_{k+1}(x_i)) (sampling importance resampling).  The mean exchange probability
 * between the two states' samples checks the spacing.  These are the device reductions of those
 * steps; the host chooses parameters and time steps.  All comps arrays are [N][4] double
 * {U_L, U_I, Psi_sg, Psi_g} on the device; state indices refer to the state table.
 * Errors: E_STATE (no states, or no ligand when configurations are gathered), E_INVALID (N < 1,
 * state index out of range, bad pointers). */

/* Population standard deviations over N samples at state k: sigma[0..3] (host) =
 * {sigma[U_L + U_I], sigma[Psi_sg], sigma[Psi_g], sigma[u_k]}, u_k the reduced energy.  FP64.
 * Synchronises. */
algdock_status algdock_state_statistics(algdock_ctx* ctx, int64_t N, const double* comps, int32_t k, double* sigma);

/* n_out (<= 1024) draws with replacement from the N samples, with weights exp(u_from - u_to): draw
 * j takes the 53-bit uniform of Philox4x32-10 counter {j, 0, counter, 6} keyed by seed, and the
 * first sample whose running weight (index order, relative to the largest) exceeds u times the
 * total.  idx [n_out] int64 (device, may be NULL) receives the indices; if x_in ([N][n_atoms][3]
 * float, device) is given, the chosen configurations are copied to x_out ([n_out][n_atoms][3]). */
algdock_status algdock_resample(algdock_ctx* ctx, int64_t N, const double* comps, int32_t k_from, int32_t k_to,
                                int32_t n_out, uint64_t seed, uint32_t counter, const float* x_in, float* x_out,
                                int64_t* idx);

/* Mean over the N pairs (i-th sample of comps_a at state ka, i-th of comps_b at state kb) of the
 * exchange probability min(1, exp(u_a(x_a) + u_b(x_b) - u_a(x_b) - u_b(x_a))), Eq. (repXacc),
 * into *p (host).  FP64.  Synchronises. */
algdock_status algdock_mean_pacc(algdock_ctx* ctx, int64_t N, const double* comps_a, const double* comps_b, int32_t ka,
                                 int32_t kb, double* p);

/* The scalar steps of protocol initialization ("Initialization"), host arithmetic without a
 * context.  A leg's states are placed one thermodynamic-length step apart from the standard
 * deviations that algdock_state_statistics returns.
 * Warming leg: T_next = min(T_end, T + speed k_B T^2 / sigma[U_S]) (T_end if sigma[U_S] = 0). */
algdock_status algdock_next_temperature(double T, double sigma_U, double speed, double T_end, double* T_next);
/* Coupling leg: alpha_next = min(1, alpha + speed / rate) with rate = |alpha_sg'| sigma[Psi_sg] /
 * (k_B T) + |alpha_g'| sigma[Psi_g] / (k_B T) + |T_T - T_H| sigma[u] / T at T = T(alpha) =
 * T_H + (T_T - T_H) alpha, the derivatives of the weights of Eq. (protocol) (1 if rate = 0). */
algdock_status algdock_next_alpha(double alpha, double sigma_sg, double sigma_g, double sigma_u, double speed,
                                  double T_T, double T_H, double* alpha_next);
/* Time-step rule: HMC acceptance above 0.8: +0.125 fs; below 0.1: -0.5 fs; below 0.4: -0.25 fs;
 * the result kept in [0.1, 5] fs. */
algdock_status algdock_adapt_dt(double dt, double acceptance, double* dt_next);
/* State insertion between cycles ("Equilibration and production"): after every neighbour pair
 * (k, k+1) of a leg whose exchange acceptance accepts[k] / attempts[k] is below threshold (pairs
 * never attempted are kept), a state at the midpoint of the leg's parameter: the geometric mean
 * temperature on the warming leg (alpha NaN), the mean alpha with T(alpha) on the coupling leg; its
 * time step is the smaller of the pair's.  Outputs (capacity >= 2K - 1): the new ladder
 * (T_out, alpha_out, dt_out [*K_out]) and lower [*K_out]: -1 for a kept state, else the index of
 * the inserted state's lower neighbour in the new ladder. */
algdock_status algdock_insert_states(int32_t K, const double* T, const double* alpha, const double* dt,
                                     const int64_t* attempts, const int64_t* accepts, double threshold, double T_T,
                                     double T_H, int32_t capacity, int32_t* K_out, double* T_out, double* alpha_out,
                                     double* dt_out, int32_t* lower);

/* ---------------------------------------------------------------- multi-ligand batches
 * Many ligands of uneven size against one set of grids and one state table, every replica of every
 * ligand in one HMC launch per atoms-per-lane class (no counterpart in the paper, which runs one
 * ligand per job; each replica's trial is the one of algdock_hmc_cycle, "Sampling").  Replicas
 * of one ligand that are consecutive in the replica order share blocks; a block stages its
 * ligand's tables once.  Launch classes: 0: <= 32 atoms; 1: 33-64 atoms whose per-pair table fits
 * 16-replica blocks of the batch kernel (its dynamic shared memory plus the kernel's own static
 * shared memory within the device's per-block limit; the one-ligand kernel then stages the table
 * too); 2: the other 33-64-atom ligands; 3: 65-96 atoms. */

/* Load n_ligands ligands (each validated as by algdock_ligand_load) with one restraint.  Replaces
 * any earlier batch and its layout; the single-ligand state (algdock_ligand_load) is untouched. */
algdock_status algdock_batch_load(algdock_ctx* ctx, int32_t n_ligands, const algdock_ligand* ligands,
                                  const algdock_restraint* rest);

/* Replica layout: replica r runs ligand lig_of[r] (host int32 [n_rep]); positions are stored
 * x_stride atoms apart ([n_rep][x_stride][3] float, only the first n_atoms of each used).  Builds
 * the work lists (runs of consecutive replicas of one ligand, longest blocks first) with a default
 * launch shape per class (the first candidate of algdock_batch_tune whose shared memory, with the
 * kernel's static shared memory, fits the device's per-block limit).
 * uniform != 0 runs every replica in the 65-96-atom class shape (the uniform baseline of a
 * batch).  ALGDOCK_E_INVALID if a ligand's tables exceed shared memory. */
algdock_status algdock_batch_layout(algdock_ctx* ctx, int64_t n_rep, const int32_t* lig_of, int32_t x_stride,
                                    int32_t uniform);

/* One HMC trial for every replica of the batch, as algdock_hmc_cycle (same Philox counters, with
 * replica index rep_offset + r).  The classes run on the context's side streams, forked from and
 * joined to its stream, so that a graph captured on that stream holds them as parallel branches.
 * Device arrays: state_of [n_rep], x [n_rep][x_stride][3], comps [n_rep][4], dH, acc (may be NULL),
 * counters (may be NULL). */
algdock_status algdock_batch_hmc_cycle(algdock_ctx* ctx, const int32_t* state_of, float* x, double* comps,
                                       double* dH, uint8_t* acc, int32_t n_steps, uint64_t seed, uint64_t cycle,
                                       int64_t rep_offset, int64_t* counters);

/* Launch shapes (for tests and tuning reports).  algdock_hmc_shape: the one-ligand HMC kernel's
 * replicas per block and 1 if it stages the per-pair table (host int32[2]).  algdock_batch_shapes:
 * the same per batch class (host int32 [4][2]; 0 for an empty class).  The pair-table and the
 * pair-type kernels round differently; the replicas per block do not change a replica's
 * arithmetic. */
algdock_status algdock_hmc_shape(algdock_ctx* ctx, int32_t* shape);
algdock_status algdock_batch_shapes(algdock_ctx* ctx, int32_t* shapes);

/* Autotuner over the launch shape of each class (classes 0, 1: replicas per block 16 or 8 with
 * the pair table staged, or 4 without; class 2: 8 with the table or 4 without; class 3: 4 or 8
 * without).  The objective is the whole batch launch, classes overlapped as in production: one
 * pass of coordinate descent, each class in turn trying its candidates with the others held, each
 * the median of n_timed launches (after one warm-up, CUDA events) from a scratch copy of x; a
 * candidate replaces the incumbent only if 2 % faster.  chosen (host
 * int32 [4][2], may be NULL): replicas per block and 1 if the table is staged, per class (0 =
 * class empty); ms (host float, may be NULL): the chosen shapes' time per launch.  x is not
 * modified.  Allocates scratch; synchronises. */
algdock_status algdock_batch_tune(algdock_ctx* ctx, const int32_t* state_of, const float* x, int32_t n_steps,
                                  int32_t n_timed, int32_t* chosen, float* ms);

/* ---------------------------------------------------------------- end points (target force field)
 * The thermodynamic cycle starts and ends in a target force field that differs from the sampling
 * force field ("Thermodynamic Cycle"); samples of milestones B and D are postprocessed in it and
 * f_AB and f_DE are estimated by free energy perturbation ("Estimation", Zwanzig 1954).  Here the
 * target force field differs from the sampling one in what the paper names as the key difference
 * apart from solvation: receptor-ligand interactions are computed directly instead of by grid
 * interpolation (there is no implicit solvent in either). */

/* Receptor atoms for the target interaction (host or device double arrays: xyz [n_rec][3],
 * rstar, eps (>= 0), q [n_rec]); copied to the context, which owns them.  n_rec = 0 is allowed
 * (the interaction is then 0).  ALGDOCK_E_NUMERIC for a non-finite or negative parameter. */
algdock_status algdock_receptor_load(algdock_ctx* ctx, int32_t n_rec, const double* rec_xyz, const double* rec_rstar,
                                     const double* rec_eps, const double* rec_q);

/* Receptor-ligand interaction of the target force field for N configurations: the grid sums of
 * algdock_grids_build taken at each ligand atom's own position and weighted by its factors,
 *   psi_T = sum_i [ sqrt(A_i) LJr(x_i) + sqrt(B_i) LJa(x_i) + q_i elec(x_i) ],
 * the same energy function as the hard grids without the interpolation (so that
 * U_T(r_RL) - U_T(r_L) - Psi_g(r_L) = psi_T - Psi_g, the exponent of the paper's reweighting of
 * milestone D samples, Eq. (reweighing_interact)).  x: device float [N][n_atoms][3] of the loaded
 * ligand; psi: device double [N] (kcal/mol).  Each pair term in FP32, sums over receptor tiles and
 * over atoms in FP64; deterministic.  Needs algdock_ligand_load and algdock_receptor_load. */
algdock_status algdock_target_interaction(algdock_ctx* ctx, int64_t N, const float* x, double* psi);

/* Zwanzig free energy perturbation over N samples of the sampling state:
 *   du_n = beta (u_target[n * stride_target] - u_sampling[n * stride_sampling]),
 *   f = -ln (1/N) sum_n exp(-du_n)   (reduced units: the target's free energy minus the sampler's).
 * u_sampling may be NULL (0); beta = 1 for energies already reduced.  For f_DE pass psi_T from
 * algdock_target_interaction and Psi_g (column 3 of the components, stride 4) at beta_T.
 * result (host double[4]): f; its first-order standard error for independent samples,
 * sqrt((N / n_eff - 1) / (N - 1)) (NaN for N = 1); the Kish effective sample size
 * n_eff = (sum w)^2 / sum w^2 of the weights w = exp(-du); the smallest du.  du = +inf has weight 0;
 * NaN or -inf gives ALGDOCK_E_NUMERIC (result still written).  FP64 log-sum-exp in a fixed
 * reduction order (deterministic).  Device arrays; synchronises. */
algdock_status algdock_fep(algdock_ctx* ctx, int64_t N, const double* u_target, int64_t stride_target,
                           const double* u_sampling, int64_t stride_sampling, double beta, double* result);

/* ---------------------------------------------------------------- learned pose proposal
 * An extension of the paper's external-coordinate moves ("Sampling": a random rotation about the
 * centre of mass and a Gaussian translation, Metropolis-tested): a network proposes rigid-body and
 * torsion increments d = (t[3] A, w[3] rad axis-angle, d_tau[T] rad), the move
 * Apply(x, d) = Rigid(d_r/2) . Tor(d_tau) . Rigid(d_r/2) satisfies Apply(Apply(x, d), -d) = x with
 * unit Jacobian, and the move is accepted with min(1, exp(-(u_k(x') - u_k(x))) q(-d|x') / q(d|x)),
 * which keeps every state's Boltzmann distribution exact whatever the network.
 *  - Torsions: root atom 0; a bond is rotatable if both atoms have >= 2 neighbours; the first
 *    T = min(16, #rotatable) in bond order are moved (the side away from the root).
 *  - Features (64): (COM - site)/d0; unit vectors COM -> atom 0 and COM -> atom n-1; (cos, sin) of
 *    the T dihedrals; alpha_sg, alpha_g, 300/T_k; asinh(component/10) of the four components; 0.
 *  - Network: 64 -> 256 -> 256 -> 256 (ReLU) -> 360 = an 8-component diagonal Gaussian mixture over
 *    the 22 (= 6 + 16) dimensions: [0,8) logits, [8,184) means [c][22], [184,360) raw log-sigma
 *    [c][22], log sigma = -2 + 4 tanh(raw / 4); only the first 6 + T dimensions are used.
 *  - Parameters: one FP32 buffer of ALGDOCK_MLP_NPARAMS floats, W1 [256][64], b1 [256], W2
 *    [256][256], b2, W3 [256][256], b3, W4 [360][256], b4 [360] (weights row-major [out][in]), and
 *    a BF16 copy of the four weight matrices (ALGDOCK_MLP_NWEIGHTS, same order).  Matrix products
 *    run on the tensor cores in BF16 with FP32 accumulation; hidden activations are stored in BF16.
 *  - Random numbers: Philox counter {draw, replica, cycle * n_moves + move, 4}: draw d < 22 the
 *    normal of dimension d, draw 100 the mixture component, draw 101 the acceptance uniform. */
enum {
  ALGDOCK_MLP_NFEAT = 64,
  ALGDOCK_MLP_NHID = 256,
  ALGDOCK_MLP_NOUT = 360,
  ALGDOCK_MLP_DMAX = 22,
  ALGDOCK_MLP_NWEIGHTS = 64 * 256 + 256 * 256 + 256 * 256 + 256 * 360,
  ALGDOCK_MLP_NPARAMS = 64 * 256 + 256 + 256 * 256 + 256 + 256 * 256 + 256 + 256 * 360 + 360
};

/* Number of moved torsions T of the loaded ligand (host call). */
algdock_status algdock_learned_ntorsions(algdock_ctx* ctx, int32_t* T);

/* Features of N poses: state_of [N] int32, x [N][n_atoms][3] float, comps [N][4] double (the
 * components of x); feat [N][64] float out. */
algdock_status algdock_learned_features(algdock_ctx* ctx, int64_t N, const int32_t* state_of, const float* x,
                                        const double* comps, float* feat);

/* Training targets: the move taking pose x to pose y (translation of the centre of mass, rotation
 * of the frame of atoms 0 and n-1, wrapped torsion differences).  x, y [N][n_atoms][3] float;
 * delta [N][22] float out (unused dimensions 0). */
algdock_status algdock_pose_delta(algdock_ctx* ctx, int64_t N, const float* x, const float* y, float* delta);

/* Network outputs for N feature rows: params FP32 [NPARAMS] (biases read from it), wbf16 [NWEIGHTS]
 * (uint16 BF16 bits); feat [N][64] float; out [N][360] float. */
algdock_status algdock_mlp_forward(algdock_ctx* ctx, const float* params, const uint16_t* wbf16, int64_t N,
                                   const float* feat, float* out);

/* Gradient of the mean negative log-density of the targets, -(1/N) sum_n log q(delta_n | feat_n),
 * over the first D dimensions: grad [NPARAMS] float out (FP32), loss (device float, may be NULL). */
algdock_status algdock_mlp_grad(algdock_ctx* ctx, const float* params, const uint16_t* wbf16, int64_t N,
                                const float* feat, const float* delta, int32_t D, float* grad, float* loss);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on params from grad; m, v [NPARAMS] moments;
 * step >= 1; refreshes the BF16 copy wbf16. */
algdock_status algdock_mlp_adam(algdock_ctx* ctx, float* params, uint16_t* wbf16, const float* grad, float* m, float* v,
                                int32_t step, float lr);

/* The tensor-core GEMM of the network (tcgen05 with tensor-memory accumulators, operands by TMA;
 * no counterpart in the paper): C = epi(A . B^T) with A [M][K] (row stride lda) and B [N][K] (ldb)
 * BF16 bit patterns, device, 16-byte aligned, lda and ldb multiples of 8; C [M][ldc] device.
 * epilogue 0: FP32; 1: FP32 + bias[N]; 2: BF16 max(0, . + bias[N]); 3: BF16, zero where
 * mask[M][ldm] (BF16) <= 0.  n_split > 1 (epilogue 0 only) splits K into FP32 partial products at
 * C + z M ldc, z < number of slices.  Synchronises; ALGDOCK_E_CUDA if a bounded wait of the kernel
 * ran out.  algdock_mlp_grad takes this path from 4096 rows and algdock_mlp_forward from 8192
 * (and they then synchronise too). */
algdock_status algdock_gemm_bf16(algdock_ctx* ctx, int32_t M, int32_t N, int32_t K, const uint16_t* A, int32_t lda,
                                 const uint16_t* B, int32_t ldb, void* C, int32_t ldc, int32_t epilogue,
                                 const float* bias, const uint16_t* mask, int32_t ldm, int32_t n_split);

/* n_moves learned proposals for each of n_rep replicas at its state (state_of), each accepted or
 * rejected as above in FP64.  n_torsions limits the moved torsions to the first
 * min(T, n_torsions) (negative: all T); the mixture then covers 6 + that many dimensions, and
 * n_torsions = 0 gives rigid-body moves only (the paper's external-coordinate moves, with a learned
 * proposal).  x and comps (the components of x) are updated in place; accepted [n_rep] int32 (may
 * be NULL) is added to; counters as for algdock_hmc_cycle (may be NULL). */
algdock_status algdock_propose_learned(algdock_ctx* ctx, const float* params, const uint16_t* wbf16, int64_t n_rep,
                                       const int32_t* state_of, float* x, double* comps, int32_t n_moves,
                                       int32_t n_torsions, uint64_t seed, uint64_t cycle, int64_t rep_offset,
                                       int32_t* accepted, int64_t* counters);

/* MBAR sharded over samples, for runs whose samples are spread over processes (one per GPU).  In
 * the self-consistent equation above the sample sum of each state splits into per-process sums,
 * while log D_n = ln sum_k N_k exp(f_k - u_kn) stays local to its sample.  One iteration is:
 * algdock_mbar_partials on every process, one exchange of the K (max, sum) pairs between them, and
 * algdock_mbar_update on every process with the pairs in the same (rank) order, which gives every
 * process the same f.  The iteration count and the stopping rule are the caller's (as in
 * algdock_mbar: stop when delta < tol). */

/* This process's pairs: pairs [K][2] (host, out) with sum_n exp(-u_in - log D_n) = pairs[i][1] *
 * exp(pairs[i][0]) over its N samples (max -inf, sum 0 for a state with none).  u_kn [K][N] double
 * (device; may be NULL if N == 0), N_k [K] int64 (host): the counts over ALL processes; f [K]
 * (host): the current estimate.  precision_mode 0 or 1 as for algdock_mbar.  Synchronises. */
algdock_status algdock_mbar_partials(algdock_ctx* ctx, int32_t K, int64_t N, const double* u_kn, const int64_t* N_k,
                                     const double* f, int32_t precision_mode, double* pairs);

/* Host arithmetic, no context: merges each state's n_parts pairs (pairs [n_parts][K][2], merged
 * in that order), f_i = -(M + ln S), gauge f_0 = 0, into f_new [K]; *delta = max_i |f_new - f_old|. */
algdock_status algdock_mbar_update(int32_t K, int32_t n_parts, const double* pairs, const double* f_old,
                                   double* f_new, double* delta);

/* ---------------------------------------------------------------- checkpoint and resume
 * The paper stores each stage's data between cycles so that a calculation interrupted on a shared
 * machine restarts where it stopped ("Stages"; "Equilibration and production").  A checkpoint
 * holds the context's state table (T, alpha and every state's time step, as last set by
 * algdock_states_set), the run's seed and next cycle, a fingerprint (CRC-32) of the loaded ligand
 * and lattice descriptor, and the caller's named arrays: whatever the run keeps between cycles
 * (positions, components, state permutations, exchange counters, stored components).  The Philox
 * counters of every step are functions of (seed, cycle, replica), so a run continued from a
 * checkpoint repeats the uninterrupted run bit for bit.
 * Format: one file, little-endian, "ALGDCKPT", version 1, sizes, the state table, the arrays (name
 * up to 31 bytes, dtype, count, data) and a CRC-32 trailer over the whole file.  The file is
 * written to a temporary name beside path and renamed over path.  Grids and ligand are inputs,
 * not state: load them before algdock_checkpoint_load. */
typedef enum { ALGDOCK_F32 = 1, ALGDOCK_F64 = 2, ALGDOCK_I32 = 3, ALGDOCK_I64 = 4, ALGDOCK_U8 = 5 } algdock_dtype;
typedef struct {
  char name[32];  /* NUL-terminated, unique within one checkpoint */
  int32_t dtype;  /* algdock_dtype */
  int64_t count;  /* elements */
  void* data;     /* host or device; read by save, written by load */
} algdock_array;

/* Saves ctx's state table and fingerprints (ctx may be NULL: none are stored), seed, cycle and the
 * n_arrays arrays to path.  Synchronises ctx's stream first.  ALGDOCK_E_INVALID: bad or duplicate
 * names, unknown dtype, negative count, or the file cannot be written. */
algdock_status algdock_checkpoint_save(algdock_ctx* ctx, const char* path, uint64_t seed, uint64_t cycle,
                                       int32_t n_arrays, const algdock_array* arrays);

/* Reads path, checks magic, version, sizes and the CRC (ALGDOCK_E_INVALID on any mismatch: a
 * corrupt or truncated file changes nothing), then: with ctx, checks that the context's loaded
 * ligand and lattice match the checkpoint's fingerprints (ALGDOCK_E_STATE otherwise) and restores
 * the state table as algdock_states_set would; fills each array whose data is non-NULL from the
 * array of the same name, which must exist with the same dtype and count (ALGDOCK_E_INVALID
 * otherwise); for an array with data == NULL writes the file's dtype and count (count -1 if
 * absent) instead, so that a caller can size its buffers first.  seed and cycle (may be NULL)
 * receive the stored values.  ctx may be NULL (host arrays only, no state table). */
algdock_status algdock_checkpoint_load(algdock_ctx* ctx, const char* path, uint64_t* seed, uint64_t* cycle,
                                       int32_t n_arrays, algdock_array* arrays);

/* MBAR without any device allocation.  The paper has no counterpart: this is a service of this
 * library for callers that cannot call cudaMalloc - for example a host framework whose caching
 * allocator owns all device memory and forbids direct allocations, or a service that reserves its
 * whole memory budget at start-up.  Same arguments, arithmetic and results as algdock_mbar for
 * precision modes 0 and 1, but the solver's scratch is a fixed 8 MiB array in the library's own
 * device memory (every GPU that loads the library holds it until the process exits); the call
 * itself allocates nothing and does not use the context's own MBAR scratch.
 *  - precision_mode 2 is rejected (ALGDOCK_E_INVALID with its own message): its FP32 copy of
 *    u_kn (K*N*4 bytes) does not fit the fixed array.  K above 65535 is rejected as well.
 *  - Sizes whose scratch exceeds 8 MiB (about 8 bytes per sample plus 16 bytes per state and
 *    chunk of 8192-32768 samples, e.g. N up to ~1e6 samples for K = 128) are rejected with
 *    ALGDOCK_E_INVALID and a message naming the bytes needed.
 *  - The first call on a device looks up the array's device address (once per device, with that
 *    device current) and keeps it for the life of the process; make that first call before any
 *    stream capture.  The kept address does not survive cudaDeviceReset: a process that resets
 *    the device must not call this entry point afterwards.
 *  - Every call on a device shares the one array, which keeps the last call's contents (each call
 *    re-initialises what it reads).  Calls whose work overlaps on the GPU (from several host
 *    threads or streams) race on it: serialise them. */
algdock_status algdock_mbar_noalloc(algdock_ctx* ctx, int32_t K, int64_t N, const double* u_kn, const int64_t* N_k,
                                    double tol, int32_t max_iter, int32_t precision_mode, double* f_k,
                                    int32_t* iters);

#ifdef __cplusplus
}
#endif
#endif /* ALGDOCK_H */
