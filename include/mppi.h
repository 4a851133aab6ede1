/*
 * mppi.h -- C ABI of libmppi, a GB300 (sm_103a) implementation of one MPPI
 * solve of the reference-free drone-racing controller of arXiv 2509.14726
 * ("Rethinking Reference Trajectories in Agile Drone Racing: A Unified
 * Reference-Free Model-Based Controller via MPPI").
 *
 * One solve (Algorithm 1, one pass of the while loop):
 *   sample   U^m = U* + dU^m, du ~ N(0, Sigma)            Sec. III-B, Eq. 3
 *   roll out every U^m through the quadrotor model         Sec. III-A, Eq. 2
 *   score it: gate progress (Eq. 6/7, Sec. IV-A), contouring (Eq. 9) or
 *             trajectory tracking (Eq. 8, Sec. IV-B)
 *   weight   w_m = exp(-J_m / lambda) / sum_i exp(-J_i / lambda)   Eq. 4
 *   update   U* = sum_m w_m U^m; apply u0*; warm start     Eq. 5, Sec. III-B
 * The problem it solves is the receding-horizon OCP of Eq. 1.
 *
 * Conventions.  All structs are plain data; every pointer argument is a
 * HOST pointer unless its name starts with d_ (device pointer).  Units: SI,
 * thrust in N, rates in rad/s, world z up, gravity (0, 0, -g).  State
 * x = [p(3), v(3), q(4, Hamilton, scalar first, body to world), w(3, body)];
 * input u = [collective thrust, body-rate command (3), progress
 * acceleration (contouring only)].  Streams are cudaStream_t passed as void*
 * (NULL = legacy default stream).
 *
 * Errors.  Every call returns an mppi_status; nothing throws across the ABI.
 * mppi_last_error() returns a thread-local message for the last failure.
 * A handle is not thread-safe: calls on one handle must be serialised by the
 * caller (different handles may be used from different threads).  The same
 * holds for an explicit batch plan (mppi_batch_*) and for the handles it
 * holds; mppi_solve_batch's internal plan cache is safe to call from several
 * threads.
 *
 * Ownership.  mppi_create deep-copies model, params and track into device
 * memory owned by the handle; the caller keeps ownership of everything it
 * passes in.  mppi_destroy releases the handle's device memory.
 */
#ifndef MPPI_H_
#define MPPI_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------------ */
/* status codes                                                              */
/* ------------------------------------------------------------------------ */
typedef enum {
  MPPI_OK = 0,
  MPPI_ERR_ARG = 1,          /* invalid argument (null, size, NaN x0, ...) */
  MPPI_ERR_OOM = 2,          /* device or pinned allocation failed */
  MPPI_ERR_CUDA = 3,         /* a CUDA runtime call failed */
  MPPI_ERR_TIMEOUT = 4,      /* a bounded device wait gave up */
  MPPI_ERR_NOT_ADMITTED = 5, /* serving: request refused by admission */
  MPPI_WARN_DEGENERATE = 6   /* every cost non-finite: nominal kept */
} mppi_status;

enum { MPPI_MODEL_CTBR = 0, MPPI_MODEL_ROTOR_RATE = 1 };
enum { MPPI_OBJ_GATE = 0, MPPI_OBJ_CONTOUR = 1, MPPI_OBJ_TRACK = 2 };
enum { MPPI_NOISE_F32 = 0, MPPI_NOISE_BF16 = 1 };
/* where the normals of Eq. 3 are drawn, all with the same Philox /
 * Box-Muller arithmetic on the same counters (bit-identical draws):
 *   KERNEL: a Philox pass before the rollout stores them; the rollout loads
 *           them, and the update (Eq. 5) loads them again;
 *   FUSED:  the rollout draws them itself and stores them for the update and
 *           the diagnostics;
 *   REGEN:  the rollout draws them and the update draws them again; nothing
 *           is stored (no noise memory: mppi_get_noise / mppi_set_noise
 *           return MPPI_ERR_ARG; needs MPPI_NOISE_F32);
 *   SMEM:   the rollout draws them and keeps its block's normals in shared
 *           memory, where the update reads them: one launch, no noise memory
 *           and no round trip to L2 in the update.  For small, latency-bound
 *           solves: the block needs 16 N_cap x (block x samples_per_thread)
 *           bytes more shared memory (20 for contouring), at most 200 KB
 *           in all (MPPI_ERR_ARG beyond); mppi_get_noise / mppi_set_noise
 *           return MPPI_ERR_ARG;
 *   AHEAD:  the Philox pass of KERNEL, run after each single solve
 *           (mppi_solve, mppi_solve_async) for the next iteration's counters,
 *           behind the event that u0 waits for: a controller that solves once
 *           per control period does not wait for its draw.  The draws and
 *           every result are those of KERNEL, bit for bit.  After a solve,
 *           mppi_get_noise returns the normals the next solve will use.  A
 *           change of shape, mppi_import_state or a batch solve (which draws
 *           before its rollout, as KERNEL does) makes the next single solve
 *           draw first again.  A solve, mppi_set_noise or a batch on
 *           another stream waits for the pending draw (an event); inside a
 *           stream capture it does not, so capture a handle's solves on one
 *           stream.  Not for the server or the allocation-free solve
 *           (MPPI_ERR_ARG). */
enum {
  MPPI_NOISEGEN_KERNEL = 0,
  MPPI_NOISEGEN_FUSED = 1,
  MPPI_NOISEGEN_REGEN = 2,
  MPPI_NOISEGEN_SMEM = 3,
  MPPI_NOISEGEN_AHEAD = 4
};
/* accumulation of the K-sample weighted update sum (Eq. 5) */
enum { MPPI_ACC_KAHAN32 = 0, MPPI_ACC_F64 = 1, MPPI_ACC_F32 = 2 };
enum { MPPI_RULE_OFF = 0, MPPI_RULE_TIME_ALIGNED = 1, MPPI_RULE_SAME_INDEX = 2 };
/* warm start of the next solve (Sec. III-B): shift the new sequence by one
 * step and repeat its last row, or keep the complete sequence (the literal
 * reading) */
enum { MPPI_WARM_SHIFT = 0, MPPI_WARM_KEEP = 1 };

#define MPPI_NX 13
#define MPPI_NU 5
#define MPPI_MAX_N 128     /* longest horizon a handle may use */
#define MPPI_MAX_GATES 64  /* most gates a track may have */
#define MPPI_MAX_SPT 8     /* most samples one rollout thread may run */

/* Quadrotor model (Eq. 2).  kind selects the input parameterisation:
 *   MPPI_MODEL_CTBR: u = (collective thrust, body-rate command); body-rate
 *     loop tau = J k_omega (w_cmd - w);
 *   MPPI_MODEL_ROTOR_RATE: u = dT_s/dt, the rates of the four rotor thrusts
 *     (Eq. 2 as printed).  The thrusts are state: they follow T + u t over a
 *     step and saturate in [thrust_min, thrust_max]; collective thrust =
 *     T1+T2+T3+T4, torque = (l/sqrt2 (T1+T2-T3-T4), l/sqrt2 (-T1+T2+T3-T4),
 *     c_tau (T1-T2+T3-T4)).  x0 stays 13-D: the rotor thrusts at x0 are the
 *     handle's own integrated commands (hover thrust until set, see
 *     mppi_set_rotor_thrusts).  u_min / u_max bound the rates; k_omega is
 *     unused.  Needs MPPI_NOISE_F32 storage. */
typedef struct {
  int32_t kind;
  float mass;         /* kg */
  float inertia[3];   /* diagonal of J, kg m^2 */
  float gravity;      /* m/s^2 */
  float k_omega;      /* body-rate loop gain, 1/s */
  float drag[3];      /* diagonal of D in Eq. 2 (0 = no drag) */
  float u_min[5];     /* input box: thrust, w_cmd x3, progress accel */
  float u_max[5];
  float omega_max;    /* body-rate bound of the feasibility penalty */
  float z_floor;      /* altitude floor of the feasibility penalty */
  float arm;          /* rotor model: arm length l, m */
  float c_tau;        /* rotor model: rotor drag-torque coefficient, m */
  float thrust_min;   /* rotor model: per-rotor thrust range, N */
  float thrust_max;
} mppi_model_t;

/* Sampling, objective and weighting parameters (Eq. 3-9, Table I). */
typedef struct {
  int32_t objective;  /* MPPI_OBJ_* */
  int32_t K;          /* samples (the paper's M) */
  int32_t N;          /* horizon steps (the paper's K) */
  float dt;           /* s; also the control period (warm start shifts 1 step) */
  float lambda;       /* temperature of Eq. 4 */
  float sigma[5];     /* diagonal of Sigma (Eq. 3) */
  uint32_t seed;      /* Philox key word 0 */
  uint32_t drone_id;  /* Philox key word 1 */
  float w_limit;      /* feasibility penalty weight */
  float q_near;       /* Q_near of Eq. 7 */
  float r_near;       /* distance threshold of Q_near, m */
  int32_t temporal_rule; /* MPPI_RULE_*: gate-pass consistency rule */
  float q_lag, q_cont;   /* Eq. 9 lag / contouring weights */
  float q_omega[3];      /* Eq. 9 body-rate weights */
  float r_dv, r_dthrust; /* Eq. 9 progress-accel and thrust-change weights */
  float mu;              /* Eq. 9 progress reward */
  float v_theta_max;     /* Eq. 9 progress-speed bound */
  float theta_back, theta_ahead; /* window of the path projection, m */
  float Q[13], QN[13];   /* Eq. 8 state / terminal weights */
  float R[4];            /* Eq. 8 input weights (about hover thrust) */
  int32_t noise_dtype;   /* MPPI_NOISE_*: storage of the sampled noise */
  int32_t accum;         /* MPPI_ACC_* */
  int32_t block;         /* threads per block of the rollout (0 = 128) */
  int32_t N_cap;         /* largest N later solves may use (0 = N) */
  int32_t K_cap;         /* largest K later solves may use (0 = K) */
  int32_t noise_gen;     /* MPPI_NOISEGEN_* */
  int32_t nominal_sample; /* 1: sample 0 is the unperturbed nominal (Eq. 3 with du = 0) */
  int32_t warm_start;    /* MPPI_WARM_* */
  int32_t samples_per_thread; /* rollouts one thread runs one after another, 1..8 (0 = 1):
                                 a block covers block x samples_per_thread samples, so a
                                 solve launches fewer blocks and pays the per-block setup
                                 (nominal copy, reductions, merge) fewer times */
} mppi_params_t;

/* Track: waypoints W, arc-length path P_arc and reference tau_ref
 * (the inputs of Algorithm 1).  Tables are row-major float32, host memory. */
typedef struct {
  int32_t n_gates;
  int32_t closed;        /* 1: gates repeat (laps) */
  const float* gates;    /* [n_gates][6]: centre x y z, yaw, half width, half height */
  int32_t S;             /* path nodes, uniform in arc length */
  float L;               /* path length, m (nodes L/S apart, closed) */
  const float* path;     /* [S][6]: position, unit tangent (NULL if S == 0) */
  int32_t T;             /* reference rows (periodic with period T*dt_ref) */
  float dt_ref;          /* s between reference rows */
  const float* ref;      /* [T][13]: p v q w (NULL if T == 0) */
} mppi_track_t;

typedef struct mppi_s* mppi_handle;
typedef struct mppi_batch_s* mppi_batch;

/* Fills *m / *p with the library defaults for mass 0.85 kg, inertia
 * diag(0.0025, 0.0025, 0.0043), thrust in [0, 4 m g], rates in [-10, 10]
 * rad/s, sigma (0.3 m g, 1, 1, 1, 5), lambda 1 and the cost weights listed in
 * the design notes.  Returns MPPI_ERR_ARG on NULL. */
int mppi_default_model(mppi_model_t* m);
int mppi_default_params(mppi_params_t* p, int32_t objective, int32_t K, int32_t N, float dt);

/* Creates a controller for one drone (Eq. 1 problem data: model, weights,
 * track).  The nominal starts at hover, the gate index at 0, the Philox
 * iteration at 0.  Must be called with the target device current.
 * Errors: MPPI_ERR_ARG (bad sizes: K < 1, N < 1 or > MPPI_MAX_N, n_gates < 1
 * or > MPPI_MAX_GATES for the gate objective, missing path / reference table
 * for the contouring / tracking objective), MPPI_ERR_OOM, MPPI_ERR_CUDA. */
int mppi_create(const mppi_model_t* model, const mppi_params_t* params,
                const mppi_track_t* track, mppi_handle* out);
int mppi_destroy(mppi_handle h);

/* One MPPI solve (Algorithm 1 body) from state x0 at time t0 (t0 selects the
 * tracking reference window; unused otherwise).  Enqueues the kernels on
 * `stream`, copies u0* (5 floats; the 5th is the progress acceleration for
 * contouring, 0 otherwise) to u0_out and waits only for that copy.  The
 * handle's nominal, gate index and RNG counter are updated on the device.
 * Returns MPPI_WARN_DEGENERATE (u0 = previous nominal) if every cost was
 * non-finite. */
int mppi_solve(mppi_handle h, const float x0[13], double t0, void* stream, float u0_out[5]);

/* Same solve with device-resident x0 and u0 (d_x0: 13 floats, d_u0: 5
 * floats), fully asynchronous: nothing is waited for. */
int mppi_solve_async(mppi_handle h, const float* d_x0, double t0, void* stream, float* d_u0);

/* Solves n independent drones in one launch sequence (uneven K, N and
 * objectives allowed).  x0s: [n][13], t0s: [n], u0s_out: [n][5], host.
 * The first call with a given handle list builds a plan (tile table, CUDA
 * graph); later calls with the same list reuse it.  Each handle's result is
 * the one mppi_solve would give (the per-solve reduction order does not
 * depend on the batch). */
int mppi_solve_batch(int32_t n, const mppi_handle* hs, const float* x0s, const double* t0s,
                     void* stream, float* u0s_out);

/* Explicit batch plans (what mppi_solve_batch caches internally).
 * use_graph = 1 captures the launch sequence in a CUDA graph with one
 * concurrent branch per (objective, noise type, block) group; use_graph = 2
 * captures it as one serial chain; 0 launches without a graph. */
int mppi_batch_create(int32_t n, const mppi_handle* hs, int32_t use_graph, mppi_batch* out);
int mppi_batch_solve(mppi_batch b, const float* x0s, const double* t0s, void* stream, float* u0s_out);
/* device-side form: d_x0s [n][13], d_t0s [n], d_u0s [n][5]; asynchronous.
 * With a graph plan, the first call with a given (d_x0s, d_t0s, d_u0s) set
 * captures the launch sequence on those buffers; later calls with the same
 * set launch it with no copies.  A plan keeps graphs for 4 sets; calls with
 * other sets copy through the plan's own buffers (two copies in, one out). */
int mppi_batch_solve_async(mppi_batch b, const float* d_x0s, const double* d_t0s, void* stream,
                           float* d_u0s);
int mppi_batch_destroy(mppi_batch b);

/* Tracing: runs the plan's launch sequence n_iters times WITHOUT the graph on
 * `stream`, with CUDA events between the phases, on the device-resident
 * inputs of the last mppi_batch_solve (or zeros).  Writes the mean duration
 * per iteration in ms of: [0] noise kernels, [1] rollout kernel of the gate
 * objective, [2] contouring, [3] tracking, [4] nominal rollout, [5] total.
 * Phases without work report 0.  Advances every handle's state n_iters
 * times, like n_iters solves. */
int mppi_batch_profile(mppi_batch b, int32_t n_iters, void* stream, float ms_out[6]);

/* Changes K and/or N of an existing handle (within K_cap / N_cap).  The
 * nominal keeps its first rows (the last row repeats when N grows). */
int mppi_set_shape(mppi_handle h, int32_t K, int32_t N);

/* ---------------- state access (checkpoint / resume, diagnostics) -------- */

/* Nominal U* (after the shift) [N][5]. */
int mppi_get_nominal(mppi_handle h, float* U);
/* Weighted average of the last solve before the shift (Eq. 5) [N][5]. */
int mppi_get_unew(mppi_handle h, float* U);
/* Per-sample cost of the last solve [K] (double: J is accumulated in
 * compensated float32 and exported as hi + lo). */
int mppi_get_costs(mppi_handle h, double* J);
/* Per-sample gate-progress diagnostics of the last solve: gates passed
 * inside the horizon and step of the first accepted pass (-1: none). */
int mppi_get_sample_info(mppi_handle h, int32_t* npass, int32_t* first_pass);
/* Sampled standard normals of the last solve [N][K][5] (the 5th column is
 * only filled for contouring, where steps 4j .. 4j+3 take the four normals
 * of block 1 at step 4j; BF16 storage is widened to float).  With
 * MPPI_NOISEGEN_AHEAD: the normals the next solve will use. */
int mppi_get_noise(mppi_handle h, float* Z);
/* Gates passed by each state of the last nominal rollout [N+1]. */
int mppi_get_passcnt(mppi_handle h, int32_t* passcnt);
/* Scalars of the last solve: [0] gate index at its start, [1] status,
 * [2] Philox iteration now, [3] gate index now. */
int mppi_get_info(mppi_handle h, int32_t info[4]);
/* theta0, v_theta0 used by the last contouring solve; J_min and the
 * normaliser sum of Eq. 4 (relative to J_min). */
int mppi_get_solve_scalars(mppi_handle h, double out[4]);
/* Tracking reference window of the last solve [N+1][13]. */
int mppi_get_xref(mppi_handle h, float* xref);

/* Serialises the handle's resident controller state (nominal, RNG
 * iteration, gate index, pass counts, previous x0, progress state, last
 * thrust).  With buf == NULL, *size receives the byte count. */
int mppi_export_state(mppi_handle h, void* buf, size_t* size);
int mppi_import_state(mppi_handle h, const void* buf, size_t size);
/* Rotor model: the rotor thrusts [4] (N) that the next solve starts from
 * (e.g. measured); get returns the current ones.  MPPI_ERR_ARG for a
 * collective-thrust handle. */
int mppi_set_rotor_thrusts(mppi_handle h, const float T[4]);
int mppi_get_rotor_thrusts(mppi_handle h, float T[4]);
/* The rollout kernel waits for the bulk copies that stage the nominal and
 * the path table in shared memory with a bounded wait; a wait that gives up
 * marks its block's samples invalid and the solve returns MPPI_ERR_TIMEOUT
 * (mppi_solve, mppi_batch_solve; the device status of the asynchronous
 * calls), keeping the nominal when no sample is left.  limit_ns sets that
 * wait's bound (default 2e8 ns).  unreachable = 1 is a testing switch: the
 * wait then targets a barrier that nothing completes, so it runs out; the
 * copies themselves still complete before the block goes on.  Not in the
 * paper: failure reporting of this implementation. */
int mppi_set_copy_wait(mppi_handle h, uint32_t limit_ns, int32_t unreachable);

/* Sets the absolute index of the gate the next solve targets (Sec. IV-A: the
 * gate the drone flies toward; indices keep counting past the last gate of a
 * closed track).  MPPI_ERR_ARG for a negative index; mppi_import_state
 * refuses a blob with one too. */
int mppi_set_gate_index(mppi_handle h, int32_t gate);

/* Uses caller-provided standard normals for the next solve instead of
 * Philox: d_Z is [N][K][4] float32 (or bf16 when the handle stores BF16
 * noise) plus, for contouring, d_Z5 [N][K] of the same type.  Device
 * pointers; the data is copied on `stream` before this returns.  With
 * nominal_sample set, sample 0's column is zeroed after the copy (it is the
 * unperturbed nominal).  MPPI_ERR_ARG for a handle with MPPI_NOISEGEN_REGEN
 * (it has no noise buffer). */
int mppi_set_noise(mppi_handle h, const void* d_Z, const void* d_Z5, void* stream);

/* Philox4x32-10 (Salmon et al., SC'11), run on the device with the same
 * round function the noise kernel uses: for i < n, writes the four words of
 * philox(ctr = (c0 + i, c1, c2, c3), key = (k0, k1)) to d_out[4 i ..].
 * For testing the generator; d_out is a device buffer of 4 n words. */
int mppi_philox(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                int32_t n, uint32_t* d_out, void* stream);
/* Box-Muller normals from the same stream: for i < n, four normals of
 * (sample i, step k, iteration it, block blk) with key (seed, drone). */
int mppi_normals(uint32_t seed, uint32_t drone, uint32_t k, uint32_t it, uint32_t blk, int32_t n,
                 float* d_out, void* stream);

/* Rolls out caller-given sequences with the kernel's model and RK4 step:
 * d_x0 [13], d_U [B][N][4] -> d_X [B][N+1][13].  For model tests. */
int mppi_rollout_states(const mppi_model_t* model, float dt, int32_t N, int32_t B,
                        const float* d_x0, const float* d_U, float* d_X, void* stream);
/* The same for the rotor model (Eq. 2 as printed): d_x0 [13], d_T0 [B][4]
 * start thrusts, d_U [B][N][4] thrust rates -> d_X [B][N+1][13] and the
 * thrusts d_T [B][N+1][4].  MPPI_ERR_ARG for a collective-thrust model. */
int mppi_rollout_states_rotor(const mppi_model_t* model, float dt, int32_t N, int32_t B, const float* d_x0,
                              const float* d_T0, const float* d_U, float* d_X, float* d_T, void* stream);

/* A solve for callers that cannot allocate device memory while they run.
 * The paper has no counterpart: this is an interface for integration.
 *
 * Some callers must not call cudaMalloc/cudaFree on their hot path: a control
 * loop certified to allocate only at start-up, a process whose GPU memory is
 * owned by another allocator, or a loop that cannot take the device-wide
 * synchronisation an allocation may cause.  mppi_create allocates, so those
 * callers use this call instead.  It runs the same noise and rollout kernels
 * as mppi_solve but allocates nothing: every per-solve scratch buffer lives in
 * one 16 MiB array in device memory that each GPU loading the library holds
 * until the process exits.
 *
 * It is stateless: one solve from the caller's nominal d_U [N][5] (device,
 * float32, unchanged), Philox iteration `iter` and gate index `gate`, as the
 * first solve of a fresh controller would do it with that nominal (no
 * previous x0, no pass counts of a previous nominal, no progress state).
 * Outputs: d_Unew [N][5] (the weighted average, before any shift; warm
 * starting is the caller's: shift it by one row for the next call) and d_u0
 * [5], both device memory.  model and params are host structs read during the
 * call; d_track holds DEVICE pointers to the gate / path / reference tables.
 * d_x0 is device memory [13]; t0 selects the tracking window.
 *
 * Limit: the scratch must fit in 16 MiB (about 16 K N (16 + 4 for
 * contouring) bytes of noise plus small tables: e.g. K = 8192 with N = 100,
 * or K = 16384 with N = 50); larger sizes return MPPI_ERR_ARG with the needed
 * byte count in mppi_last_error().
 *
 * Set-up: the first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and sets kernel
 * attributes; make that first call before any stream capture.  Every call on
 * a device shares the one array and leaves its contents behind; each call
 * clears what must start at zero.  Calls whose work overlaps on the GPU (two
 * streams, or two threads) race on the array and give wrong results: issue
 * them on one stream, or order them.  Asynchronous: returns after enqueueing
 * on `stream`.  Errors: MPPI_ERR_ARG (null pointer, bad sizes, scratch limit,
 * a negative gate index, a rotor-thrust-rate model: its rotor thrusts are
 * handle state), MPPI_ERR_CUDA. */
int mppi_solve_noalloc(const mppi_model_t* model, const mppi_params_t* params, const mppi_track_t* d_track,
                       const float* d_x0, double t0, const float* d_U, uint32_t iter, int32_t gate,
                       void* stream, float* d_Unew, float* d_u0);

/* ---------------- serving: continuous batching of many drones ------------ */
/* A server owns many drones' resident controller state (nominal, Philox
 * iteration, gate index, pass counts, progress state: a few KB each) and one
 * device pool of scratch memory of a fixed budget.  Solve requests from the
 * drones (each with its own K and N, up to the drone's caps) queue on the
 * host; mppi_server_step admits queued requests in arrival order while their
 * scratch (noise, costs, tile partials: about 16 K N bytes each, 20 K N for
 * contouring; about 12 K + 40 N K/block bytes with MPPI_NOISEGEN_REGEN)
 * fits in the pool's free space, and launches them as one batch
 * (the kernels of mppi_solve_batch) on the next free stream slot, so batches
 * overlap on the device while later requests keep arriving.  A drone has at
 * most one request in flight; its next request waits for the previous one.
 * mppi_server_poll returns finished requests.  Each result equals what
 * mppi_solve on a handle with the same state would give (same kernels, same
 * per-solve reduction order).  The paper has no serving layer; this is the
 * batching the GPU needs to run many controllers at their own rates. */
typedef struct mppi_server_s* mppi_server;

typedef struct {
  int64_t request;   /* id returned by mppi_server_submit */
  int32_t drone;
  int32_t status;    /* mppi_status of the solve */
  int32_t K, N;
  float u0[5];
  double t_submit;   /* mppi_clock() when submitted */
  double t_launch;   /* when its batch was launched */
  double t_done;     /* when a poll saw it finished */
} mppi_result_t;

/* Host monotonic clock in seconds (the server's timestamps). */
double mppi_clock(void);

/* max_drones: drones the server may hold; scratch_budget_bytes: device pool
 * for in-flight requests; n_slots: batches that may be in flight at once
 * (one stream each); max_batch: requests per batch.  Errors: MPPI_ERR_ARG,
 * MPPI_ERR_OOM (the pool or the staging buffers), MPPI_ERR_CUDA. */
int mppi_server_create(int32_t max_drones, size_t scratch_budget_bytes, int32_t n_slots, int32_t max_batch,
                       mppi_server* out);
/* Adds a drone (model, params with K_cap / N_cap = its largest request, and
 * track, as for mppi_create; block must be 128 or less).  Writes its id. */
int mppi_server_add_drone(mppi_server s, const mppi_model_t* model, const mppi_params_t* params,
                          const mppi_track_t* track, int32_t* drone_out);
/* Queues n requests (host arrays: drones [n], x0s [n][13], t0s [n], Ks [n],
 * Ns [n]); writes their ids (may be NULL).  A request whose K or N exceeds
 * its drone's caps, whose scratch exceeds the whole pool, or whose tiles
 * exceed what one batch holds, is refused with MPPI_ERR_NOT_ADMITTED (none of
 * the n is queued then). */
int mppi_server_submit(mppi_server s, int32_t n, const int32_t* drones, const float* x0s, const double* t0s,
                       const int32_t* Ks, const int32_t* Ns, int64_t* ids_out);
/* The same with a deadline per request (host array [n] of mppi_clock()
 * times; 0 = none): a request still queued at its deadline is not launched
 * but dropped (load shedding: a controller gains nothing from a solve whose
 * control period has passed).  Dropped requests come back from
 * mppi_server_poll with status MPPI_ERR_NOT_ADMITTED and t_launch 0. */
int mppi_server_submit_deadline(mppi_server s, int32_t n, const int32_t* drones, const float* x0s,
                                const double* t0s, const int32_t* Ks, const int32_t* Ns, const double* deadlines,
                                int64_t* ids_out);
/* Admits and launches at most one batch if a slot is free; writes how many
 * requests it launched (0 if none could be admitted).  If the transfer or a
 * launch of the batch fails, the admitted requests are handed back (scratch
 * released, drones idle, requests queued again in arrival order) and the call
 * returns MPPI_ERR_CUDA; a later step retries them. */
int mppi_server_step(mppi_server s, int32_t* launched);
/* Testing hook for that recovery path (no counterpart in the paper): the
 * next mppi_server_step that admits a batch fails on the host, before any
 * transfer or launch, as if the batch's first launch had failed. */
int mppi_server_fail_next_launch(mppi_server s);
/* Collects finished requests (up to cap) into out; writes their count. */
int mppi_server_poll(mppi_server s, mppi_result_t* out, int32_t cap, int32_t* n_out);
/* [0] queued, [1] in flight, [2] scratch bytes in use, [3] peak scratch
 * bytes, [4] batches launched, [5] requests finished, [6] drones, [7] pool bytes. */
int mppi_server_stats(mppi_server s, double out[8]);
/* Exports one drone's controller state (the mppi_export_state layout). */
int mppi_server_export_drone(mppi_server s, int32_t drone, void* buf, size_t* size);
/* Waits for everything in flight, then frees all device memory. */
int mppi_server_destroy(mppi_server s);

/* Device memory the handle holds, bytes. */
int mppi_device_bytes(mppi_handle h, size_t* bytes);
/* Device memory a handle with these params would hold, bytes. */
int mppi_estimate_bytes(const mppi_params_t* params, const mppi_track_t* track, size_t* bytes);

/* sizeof(mppi_model_t), sizeof(mppi_params_t), sizeof(mppi_track_t) as
 * compiled into the library, for binding checks.  Touches no device. */
int mppi_abi_sizes(size_t out[3]);

/* Number of kernels the library has launched since load (all entry points). */
uint64_t mppi_kernel_launches(void);

const char* mppi_last_error(void);
const char* mppi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MPPI_H_ */
