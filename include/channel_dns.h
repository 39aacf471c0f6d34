/*
 * channel_dns.h -- C ABI of the GPU channel-flow environment.
 *
 * The library advances an incompressible plane-channel flow, simulated by a
 * pseudo-spectral DNS (Fourier modes in x and z, Chebyshev polynomials in y;
 * paper Sec. 3.1), under wall blowing/suction control (paper Sec. 3.2).  One
 * environment step mirrors the paper's request cycle (Sec. 3.3): set the
 * control (CNTRL), evolve the solver several time steps (EVOLVE), return the
 * observation planes and the wall-shear reward (STATE); env_destroy ends it
 * (TERMN).
 *
 * Numerical method (the readings of the paper that the library fixes):
 *   - channel y in [-1, 1]; the action is the wall-normal velocity of the
 *     lower (no-slip) wall y = -1; the upper boundary is a no-slip wall
 *     (closed channel, top_bc = 0) or free slip (the paper's open channel,
 *     top_bc = 1);
 *   - velocity-vorticity (v, omega_y) form, 3/2-dealiased u x omega;
 *   - third-order low-storage Runge-Kutta for the nonlinear term and
 *     Crank-Nicolson for the viscous term (Sec. 3.1), coefficients
 *     gamma = (8/15, 5/12, 3/4), zeta = (0, -17/60, -5/12),
 *     alpha = beta = (gamma + zeta) / 2;
 *   - Chebyshev-tau Helmholtz solves per Fourier mode with an influence-matrix
 *     correction for the four v wall conditions;
 *   - constant flow rate: the mean pressure gradient is set every stage so
 *     that the bulk velocity stays 1.
 * Units: y in [-1, 1], bulk velocity 1, u_tau = re_tau / re_bulk; nu =
 * 1 / re_bulk (closed channel: Reynolds numbers on the half height 1) or
 * 2 / re_bulk (open channel: on its height 2).
 *
 * Conventions
 *   - All functions return 0 (CH_OK) on success or a negative CH_ERR_* code;
 *     ch_strerror() names it.  A failing call leaves no partial result the
 *     caller must free.
 *   - The library owns every device allocation it makes; the caller owns all
 *     host buffers (they must stay valid until the call returns) and every
 *     device buffer it passes in.
 *   - One thread at a time per environment handle.
 *   - Layouts are row-major C arrays.  Spectral arrays hold the kept
 *     half-spectrum: kx index 0..nx/2-1 (fastest), kz rows in FFT order
 *     0..nz/2-1, -nz/2..-1 where the -nz/2 (Nyquist) row is always zero.
 *   - A batch of B environments with identical parameters shares every
 *     launch; batched arrays carry a leading [B] dimension.
 */
#ifndef CHANNEL_DNS_H
#define CHANNEL_DNS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
#define CH_OK              0
#define CH_ERR_ARG        -1   /* invalid argument, size or parameter        */
#define CH_ERR_OOM        -2   /* device or host allocation failed           */
#define CH_ERR_BUDGET     -3   /* would exceed a memory budget               */
#define CH_ERR_DIVERGED   -4   /* non-finite wall shear: the flow blew up     */
#define CH_ERR_TIMEOUT    -5   /* a bounded wait ran out                     */
#define CH_ERR_STATE      -6   /* call not valid in the handle's state       */
#define CH_ERR_CUDA       -7   /* a CUDA runtime call failed                 */
#define CH_ERR_UNSUPPORTED -8  /* parameter combination not built            */
#define CH_PENDING         1   /* srv_poll: request not finished yet (not an error) */

/* ---- parameters ---------------------------------------------------------- */
typedef struct ch_params {
    int nx, ny, nz;          /* Fourier modes in x, Chebyshev nodes in y, Fourier modes in z
                                (nx, nz even >= 4; ny odd or even >= 9, <= 201)        */
    double lx, lz;           /* box length and width in half heights                  */
    double re_tau;           /* friction Reynolds number (sets u_tau and the sensing plane) */
    double re_bulk;          /* bulk Reynolds number U_b h / nu (> 0)                  */
    double dt;               /* time step in h / U_b                                   */
    int steps_per_action;    /* solver steps per env_step (actuation interval, Sec. 3.2) */
    double y_sense_plus;     /* sensing height in wall units; rounded up to a node (Sec. 3.2) */
    int top_bc;              /* 0: closed channel, no-slip upper wall at y = +1; 1: open
                                channel of the paper (Sec. 3.1), free-slip top: v = 0,
                                D^2 v = 0, D omega_y = 0, DU = DW = 0 at y = +1, and Re_b,
                                Re_tau based on the whole height 2 (nu = 2 / re_bulk,
                                y+ = (1 + y) re_tau / 2); built for ny <= 65, larger ny
                                return CH_ERR_UNSUPPORTED                                  */
    int precision;           /* 0: all FP64; 1: mixed -- the dealiased nonlinear term
                                (Chebyshev synthesis/analysis, padded FFTs, products)
                                in FP32, the tau solves, influence-matrix correction
                                and flow-rate update in FP64                            */
    int control;             /* 0: external action, 1: opposition control (Sec. 4.1),
                                2: on-device policy (env_set_policy)                    */
    double alpha;            /* opposition-control gain                                */
    double tau_ref;          /* reward reference wall shear; <= 0 -> u_tau^2          */
    int batch;               /* number of environments B sharing launches; <= 0 -> 1   */
    int autotune;            /* 1 (default): env_create times the candidate tile shapes of
                                the stage kernels on this grid and batch and keeps the
                                fastest; 0: size heuristic.  The candidates perform the
                                same floating-point operations per output, so the choice
                                changes speed only, never results                       */
} ch_params_t;

typedef struct ch_info {
    int j_sense;             /* Gauss-Lobatto node index of the sensing plane (0 = upper wall) */
    double y_plus_sense;     /* its height above the lower wall in wall units              */
    double nu, u_tau, tau_ref;
    size_t state_bytes;      /* bytes of one environment's serialised state                */
    size_t device_bytes;     /* device memory held by the handle                           */
    int plane_cluster;       /* CTAs of a thread-block cluster cooperating on one y-plane of
                                the nonlinear term; 0: no portable cluster holds the plane
                                (planes of 256 x 256 modes), the term runs in three passes
                                through a global scratch array (z inverse, x transforms and
                                products, z forward)                                     */
    int launches_per_step;   /* kernels launched by one env_step                            */
    int post_batched;        /* 1: the implicit half of a stage runs one thread per (mode,
                                class, component); 0: eight threads per mode on a tile  */
    int ppc_pre, ppc_post;   /* Fourier modes per CTA of the explicit and implicit halves */
    int tuned;               /* 1 if the tile shapes were chosen by timing (autotune)    */
    double tune_ms;          /* host time env_create spent timing candidates            */
    int plane_team;          /* 1: planes of 16 x 16 modes in a batch of at least four
                                planes per SM; each padded 24 x 24 plane is owned by a team
                                of 96 threads that transforms its 24-point lines in
                                registers (plane_cluster is then 1); 0 otherwise          */
} ch_info_t;

typedef struct ch_env ch_env_t;

/* Fill *p with the minimal-channel defaults of the paper's first domain
 * (16 x 65 x 16, 2.67 x 2 x 0.8, Re_tau 180, Re_b 2800, dt 0.005). */
int ch_default_params(ch_params_t* p);

/* Create B = p->batch environments on the current CUDA device.  Allocates all
 * device state and precomputes the per-mode tau factorisations.  The flow is
 * laminar Poiseuille with zero wall action until env_reset/env_set_state.
 * Errors: CH_ERR_ARG (bad sizes/parameters), CH_ERR_UNSUPPORTED,
 * CH_ERR_OOM, CH_ERR_CUDA. */
int env_create(const ch_params_t* p, ch_env_t** out);

/* Launch all further work of this handle on `stream` (a cudaStream_t; NULL
 * selects the library's own stream). */
int env_set_stream(ch_env_t* env, void* stream);

/* Laminar Poiseuille flow plus a seeded divergence-free perturbation in every
 * environment (environment e uses seed + e): SplitMix64 normals, v = s (a+ib)
 * (1-y^2)^2 and omega_y = s (c+id) (1-y^2) on modes with kx and |kz| index
 * <= kmax, s = amplitude / sqrt(#modes).  Time and wall action are zeroed. */
int env_reset(ch_env_t* env, uint64_t seed, double amplitude, int kmax);

/* One interaction for every environment of the batch, host buffers:
 *   action     [B][nz][nx] wall-normal velocity at the lower wall (ignored and
 *              may be NULL under opposition control); clipped to
 *              [-u_tau, u_tau], plane mean removed, ramped linearly from the
 *              previous action over the steps_per_action steps (Sec. 3.2);
 *   obs        [B][2][nz][nx] u and v on the sensing plane after the steps;
 *   wall_shear [B] nu dU/dy at the lower wall averaged over the steps;
 *   reward     [B] 1 - wall_shear / tau_ref (Sec. 3.2).
 * Any of obs, wall_shear, reward may be NULL.  The observations are copied
 * from the device straight into obs (one pitched copy; pinned memory lets it
 * run as a DMA, pageable memory is staged by the driver).
 * Synchronises the stream.  Returns CH_ERR_ARG without doing any work if the
 * action holds a non-finite value, and CH_ERR_DIVERGED if any wall shear is
 * not finite (outputs are still written). */
int env_step(ch_env_t* env, const double* action, double* obs,
             double* wall_shear, double* reward);

/* Same as env_step with DEVICE buffers, asynchronous on the handle's stream:
 *   d_action [B][nz][nx] (may be NULL under opposition control);
 *   d_out    [B][2 nz nx + 2]: per environment the two observation planes,
 *            then the mean wall shear and the reward.
 * No host synchronisation, no divergence check. */
int env_step_device(ch_env_t* env, const double* d_action, double* d_out);

/* Serialised state of environment `e` (host buffer of info.state_bytes):
 *   double v[ny][nz][nx/2][2]   Chebyshev coefficients of v per mode (re, im)
 *   double g[ny][nz][nx/2][2]   same for omega_y
 *   double U[ny], W[ny]         mean-flow Chebyshev coefficients
 *   double vw[nz][nx/2][2]      spectrum of the last applied wall action
 *   double t, steps             simulated time and completed solver steps */
int env_get_state(ch_env_t* env, int e, void* buf, size_t nbytes);
int env_set_state(ch_env_t* env, int e, const void* buf, size_t nbytes);

/* Same problems and result as ch_tau_helmholtz, for callers that must not
 * allocate device memory at all: hard real-time control loops (an allocation,
 * or the driver growing per-thread local memory for a new kernel, can block
 * and synchronise the device), processes whose device memory is fully owned
 * by another allocator, and hosts that only lend buffers they own.  The paper
 * has no counterpart; this is a deployment variant.
 *   - The caller passes all inputs and outputs (device pointers, as for
 *     ch_tau_helmholtz).  The work vectors live in one 16 MiB array that the
 *     library reserves on every GPU that loads it, until the process exits.
 *   - Capacity: 2 * M * 8 * mpad doubles <= 2^21, with mpad = ny/2 + 1 rounded
 *     up to even (ny = 65: M <= 3855; ny = 129: M <= 1985).  Larger requests
 *     return CH_ERR_ARG without launching; split them.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture.
 *   - All calls share the array: calls that overlap on the GPU (different
 *     streams, or host threads) race and must be serialised by the caller.
 *     Nothing in it needs to start at zero; every call writes what it reads.
 *   - No cudaMalloc, cudaFree or other allocating call is made. */
int ch_tau_helmholtz_noalloc(int ny, int M, const double* d_lam, const double* d_r,
                             const double* d_top, const double* d_bot, double* d_f,
                             void* stream);

/* Kernel timing for measurement tools.  While enabled, every launch of the
 * handle is bracketed by a pair of CUDA events on the handle's stream and
 * attributed to a class: 0 stage_pre (u, w, vorticity from v, omega_y and
 * their values at the Chebyshev nodes), 1 nonlinear plane kernel,
 * 2 stage_post (Chebyshev analysis of H, right-hand sides, tau solves),
 * 3 per-step kernels (action, wall shear, observation).
 * env_profile(env, 1) clears the totals and starts recording, (env, 0) stops.
 * env_profile_read synchronises the stream and returns the summed device
 * time (ms) and the launch count of one class since the last enable. */
int env_profile(ch_env_t* env, int enable);
int env_profile_read(ch_env_t* env, int cls, double* total_ms, int* launches);

int env_info(const ch_env_t* env, ch_info_t* info);

/* Pin the tile shapes of the two stage kernels (overriding the autotuner):
 * ppc_pre in {1, 2, 4, 8} modes per 128-thread CTA of the explicit half;
 * post_batched 0 with ppc_post in 1..8 (8 threads per mode) or 1 with
 * ppc_post in {1, 2, 4, 8, 16} (4 threads per mode).  Every shape gives
 * bit-identical results.  Waits for the handle's stream.  No counterpart in
 * the paper (a tuning control of this implementation).
 * Errors: CH_ERR_ARG (bad handle or shape, or a shape whose shared memory
 * exceeds the device limit), CH_ERR_CUDA. */
int env_set_tiles(ch_env_t* env, int ppc_pre, int ppc_post, int post_batched);

/* On-device policy (control = 2).  Sec. 3.2: one agent per wall grid point,
 * all sharing one policy that maps the observed part of the sensing plane
 * above the agent's actuator to its wall-normal velocity (learnt by DDPG,
 * whose actor is a multilayer perceptron; the paper gives no architecture).
 * At the start of every step the library evaluates, for every agent, a
 * perceptron with n_hidden ReLU layers on the u and v values of a periodic
 * wz x wx window of the current sensing plane centred on the agent, in FP32,
 * and applies the result as the wall action of the step (clipped to
 * [-u_tau, u_tau], plane mean removed, ramped from the previous action, as an
 * external action is).  The policy's input is the observation the previous
 * step returned. */
typedef struct ch_policy {
    int wz, wx;              /* odd window sides, 1..7, at most nz and nx         */
    int n_hidden;            /* 0 (linear), 1 or 2 hidden layers                   */
    int width[2];            /* hidden widths, 1..64 (width[1] used if n_hidden 2) */
    int out_tanh;            /* 1: action = u_tau tanh(y); 0: action = y           */
} ch_policy_t;

/* Set the policy.  weights (host, FP64, rounded to FP32 on upload): per layer,
 * W [out][in] row-major then the bias [out]; layer 0 has K = 2 wz wx inputs
 * x[(c wz + dz) wx + dx] = plane c (0: u, 1: v) at row (iz + dz - wz/2) mod nz
 * and column (ix + dx - wx/2) mod nx of agent (iz, ix); the last layer has one
 * output.  n_weights must be the count these sizes give.  Waits for the
 * handle's stream.  Errors: CH_ERR_ARG (sizes, count or a non-finite weight),
 * CH_ERR_STATE (handle not created with control = 2), CH_ERR_CUDA.  env_step on
 * a control-2 handle without a policy returns CH_ERR_STATE. */
int env_set_policy(ch_env_t* env, const ch_policy_t* pol, const double* weights, size_t n_weights);

/* STATE without a step (Sec. 3.3): u and v on the sensing plane of the
 * current flow, obs [B][2][nz][nx] (host), the same values env_step returns
 * after a step.  Synchronises the stream.  Errors: CH_ERR_ARG, CH_ERR_CUDA. */
int env_observe(ch_env_t* env, double* obs);

/* The wall action [B][nz][nx] of the last step before clipping and mean
 * removal: the caller's (control 0) or the policy's (control 2), host buffer.
 * Synchronises the stream.  Errors: CH_ERR_ARG, CH_ERR_STATE (control 1),
 * CH_ERR_CUDA. */
int env_get_action(ch_env_t* env, double* action);
int env_destroy(ch_env_t* env);
const char* ch_strerror(int code);

/* Host only (no GPU): write the env_reset initial state of one environment
 * into `buf` (same layout as env_get_state).  With p->top_bc = 1 (free-slip
 * top) the perturbation shapes are
 * v ~ (1+y)^2 (1-y) (2-y) / 2 and omega_y ~ (1+y) (3-y) / 4 and the mean flow is
 * the half-Poiseuille 1.5 (2s - s^2), s = (1+y)/2, which meet the free-slip
 * conditions exactly. */
int ch_seed_state(const ch_params_t* p, uint64_t seed, double amplitude, int kmax,
                  void* buf, size_t nbytes);

/* Host only: bytes of one serialised state for these parameters. */
size_t ch_state_bytes(const ch_params_t* p);

/* ---- serving: continuous batching of env steps from many actors ---------
 * Environments are grouped into classes by their parameters (everything in
 * ch_params_t except `batch`).  Each class owns one batched handle with
 * `slots_per_class` slots and its own CUDA stream, prioritised by the cost
 * of one env-step of the class (cheaper classes first, so that small
 * environments keep their latency next to large ones).  A worker thread runs
 * ticks: for each class with a free tick it takes the oldest pending request
 * of every environment not already in a running tick and advances exactly
 * those slots in one masked batched step; a class keeps up to two ticks in
 * flight, ticks of different classes overlap on the device, and requests
 * arriving during a tick join a later one.  A slot's result does not depend on the
 * other slots, so an environment steps identically alone and in any mix.
 * All srv_* functions are thread-safe. */
typedef struct ch_server ch_server_t;

typedef struct ch_srv_stats {
    uint64_t completed;      /* requests completed since creation / last reset   */
    double p50_us, p99_us, mean_us, max_us;  /* submit -> completion latency over the
                                                last 2^20 completed requests            */
    double env_steps_per_s;  /* completed / wall time since creation / last reset */
    int classes, envs, pending;
    size_t hbm_used, hbm_budget;  /* device bytes held by the class handles      */
    int worker_status;       /* last CUDA error seen by the worker (CH_OK if none) */
} ch_srv_stats_t;

/* Server with a device-memory budget for its class handles.  No GPU work yet. */
int srv_create(size_t hbm_budget_bytes, int slots_per_class, ch_server_t** out);

/* Bounded batching window, in microseconds (0, the default, up to 10^6).
 * While some of a class's environments have a request pending and others do
 * not, the class's next tick waits until every environment has one or until
 * linger_us have passed since the oldest pending request, whichever comes
 * first.  Larger ticks raise throughput when actors submit at nearly the same
 * time; a request waits at most linger_us longer.  CH_ERR_ARG out of range. */
int srv_set_linger(ch_server_t* s, int linger_us);

/* Admit one environment with the env_reset initial state (seed, amplitude,
 * kmax).  Uses a free slot of its class; otherwise creates the class, which
 * fails with CH_ERR_BUDGET if its footprint does not fit the budget (retry
 * after srv_evict).  Writes the environment id.  CH_ERR_UNSUPPORTED for
 * control = 2 (the server takes actions from its requests). */
int srv_admit(ch_server_t* s, const ch_params_t* p, uint64_t seed, double amplitude, int kmax, int* env_id);

/* Remove an environment; its queued requests complete with CH_ERR_STATE.  A
 * class with no environment left releases its device memory. */
int srv_evict(ch_server_t* s, int env_id);

/* Queue one env_step (action [nz][nx], copied before return; NULL under
 * opposition control; a non-finite value is rejected with CH_ERR_ARG).
 * Requests of one environment run in submission order. */
int srv_submit(ch_server_t* s, int env_id, const double* action, uint64_t* req_id);

/* srv_submit for n requests at once (an actor driving many environments):
 * env_ids [n]; actions holds, in order, one [nz][nx] plane for every request
 * whose environment takes external actions (NULL if none does); req_ids [n]
 * receives the ids.  Every request is checked first (unknown environment,
 * missing or non-finite action: CH_ERR_ARG) and then all are queued at once,
 * so a refused batch queues nothing. */
int srv_submit_many(ch_server_t* s, int n, const int* env_ids, const double* actions, uint64_t* req_ids);

/* Result of a request: CH_PENDING while it runs; otherwise its status, with
 * obs [2][nz][nx], wall shear, reward and the submit-to-completion latency
 * written (any output pointer may be NULL) and the request released. */
int srv_poll(ch_server_t* s, uint64_t req_id, double* obs, double* wall_shear, double* reward,
             double* latency_us);

/* srv_poll that waits up to timeout_ms; CH_ERR_TIMEOUT if still running. */
int srv_wait(ch_server_t* s, uint64_t req_id, int timeout_ms, double* obs, double* wall_shear,
             double* reward, double* latency_us);

/* Wait up to timeout_ms for n requests to finish, then release them all:
 * obs receives their [2][nz][nx] planes in order (may be NULL), wall_shear
 * and reward [n] (may be NULL), status [n] each request's status.  CH_OK once
 * all have finished (their statuses say how), CH_ERR_TIMEOUT with nothing
 * released if some are still running, CH_ERR_ARG for an unknown id. */
int srv_wait_many(ch_server_t* s, int n, const uint64_t* req_ids, int timeout_ms, double* obs, double* wall_shear,
                  double* reward, int* status);

/* State of an admitted environment (layout of env_get_state); waits for
 * its class to be idle.  srv_set_state requires no queued request. */
int srv_get_state(ch_server_t* s, int env_id, void* buf, size_t nbytes);
int srv_set_state(ch_server_t* s, int env_id, const void* buf, size_t nbytes);

/* Latency percentiles and throughput; reset != 0 restarts the counters. */
int srv_stats(ch_server_t* s, ch_srv_stats_t* stats, int reset);

/* Stop the worker, wait for running ticks, release all device memory. */
int srv_destroy(ch_server_t* s);

/* ---- single stages, exposed for unit checks ---------------------------- */

/* Dealiased nonlinear term of every environment of `env` on every
 * Gauss-Lobatto plane (3/2 rule), asynchronous on the handle's stream:
 *   d_q [B][6][ny][nz][nx/2] complex (re, im doubles): Fourier coefficients,
 *       at each node, of u, v, w, omega_x, omega_y, omega_z;
 *   d_h [B][3][ny][nz][nx/2] complex: Fourier coefficients of the kept modes
 *       of H = u x omega evaluated on the 3nx/2 x 3nz/2 grid.
 * Uses the handle's twiddle tables (and, for FP64 handles of 256 x 256
 * modes, their three-pass scratch array); allocates nothing.
 * CH_ERR_UNSUPPORTED for mixed-precision handles whose FP64 padded plane
 * does not fit a cluster's shared memory (256 x 256 modes). */
int ch_nonlinear(ch_env_t* env, const double* d_q, double* d_h);

/* Chebyshev-tau Dirichlet problems (D^2 - lam_m) f = r (coefficient rows
 * 0..ny-3), f(+1) = top_m, f(-1) = bot_m for M independent problems:
 *   d_lam [M] (>= 0), d_r [M][ny] complex, d_top/d_bot [M] complex,
 *   d_f [M][ny] complex output.  Device pointers, asynchronous on `stream`. */
int ch_tau_helmholtz(int ny, int M, const double* d_lam, const double* d_r,
                     const double* d_top, const double* d_bot, double* d_f,
                     void* stream);

#ifdef __cplusplus
}
#endif
#endif /* CHANNEL_DNS_H */
