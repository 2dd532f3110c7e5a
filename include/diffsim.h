/*
 * diffsim.h - C ABI of the batched differentiable contact-simulation step (sm_103a).
 *
 * One call advances B independent environments (a kinematic-tree robot touching a ground plane)
 * by one time step and, on request, differentiates the step.  The method is that of
 * "Highly-Efficient Differentiable Simulation for Robotics" (arXiv 2409.07107):
 *   - the symplectic-Euler impulse step  v+ = v + dt (vdot_f + M^-1 J_c^T lambda)   (Sec. 2.3, Eq. 3)
 *     with lambda read as an impulse, so that sigma = J_c v+ = G lambda + g          (Eq. 4);
 *   - the Coulomb-cone NCP with the De Saxce correction                            (Sec. 2.2, Eq. 1),
 *     solved by ADMM (Sec. 2.2) followed by Newton steps on the identified modes;
 *   - implicit differentiation of the NCP with breaking / sticking / sliding modes
 *     (Sec. 3.2, Eq. 8-10, App. A), the reduced system A X = -B(dG lambda + dg)   (Sec. 3.3, App. B),
 *     chained with the rigid-body derivatives and the contact-point terms           (Sec. 3.1, 3.4, App. C, D).
 *
 * Conventions (all arrays are caller-owned DEVICE memory unless stated; no call allocates):
 *   - state and outputs are structure-of-arrays with the environment index fastest:
 *       element (r, e) of an [R][B] array is at r * B + e;
 *   - q [nq_max][B], v and tau [nv_max][B] (FP64); rows beyond a model's nq / nv are ignored;
 *   - free-flyer q = (x, y, z, qw, qx, qy, qz), its velocity (linear, angular) in its own frame;
 *     derivatives w.r.t. q are taken w.r.t. the tangent perturbation q (+) dq (nv columns);
 *   - contact slot k of env e: body c_link[k*B+e] (-1 = unused), reference point
 *     c_point[(k*3+i)*B+e] in the body frame, sphere radius c_radius[k*B+e] (0 = corner),
 *     friction c_mu[k*B+e]; ground plane plane[i*B+e] = (nx, ny, nz, d): points x with n.x = d.
 *     A slot is active iff n.x - d - r <= 0 (x = reference point in world coordinates);
 *   - contact triplets are ordered (T1, T2, N) in the contact frame t1 = normalize(e_x - (n.e_x) n)
 *     (e_y instead of e_x when |n_x| > 0.9), t2 = n x t1, normal last;
 *   - lambda [3*ncmax][B]: contact IMPULSES per slot (0 for inactive slots);
 *   - modes [ncmax][B]: DS_MODE_* per slot;
 *   - Jacobians dv_dq, dv_dv, dv_dtau [nv][nv][B]: element (row i, col j) at (i*nv + j)*B + e;
 *   - a batch may mix models (model_id): each env reads and writes the leading nq / nv rows of
 *     the arrays for its own model; its Jacobians use the leading nv*nv rows of the [nv_max^2][B]
 *     arrays, element (i, j) at (i*nv + j)*B + e with its own model's nv.
 * All calls are asynchronous on the given stream (a cudaStream_t passed as void*, NULL = default
 * stream).  The return code reports argument and launch errors only; per-environment numerical
 * outcomes go to env_status.  Inputs are never modified.
 */
#ifndef DIFFSIM_H
#define DIFFSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DS_OK = 0,
  DS_EINVAL = -1,        /* a NULL pointer, a size out of range, an unsupported model shape   */
  DS_ECUDA = -2,         /* a CUDA runtime call or kernel launch failed                         */
  DS_ENOMEM = -3,        /* ds_model_create could not allocate the model's device copy          */
  DS_EUNSUPPORTED = -4,  /* no compiled kernel for this (bodies, dofs, contact slots) shape     */
  DS_ETOOLARGE = -5      /* batch too large for sim_step_jac_noalloc's fixed scratch           */
} ds_status;

typedef enum { DS_FP64 = 0, DS_MIXED = 1 } ds_precision;
/* The iteration of the NCP solve (Eq. 1; Sec. 2.2 names both families): DS_ADMM, the relaxed
 * ADMM with the De Saxce term; DS_PGS, projected Gauss-Seidel sweeps over the contacts (contact i
 * takes the fixed-point step of Eq. 1 on its own 3x3 block of G with step 1 / lambda_max(G_ii)).
 * Either iteration is staged with the same Newton polish and FP64 residual acceptance. */
typedef enum { DS_ADMM = 0, DS_PGS = 1 } ds_solver;
/* DS_MIXED: kinematics, contact detection, J_c, G and g, the residuals of the NCP polish, the NCP
 * residual check and the reduced implicit system in FP64; dynamics, ADMM iterations, derivative
 * passes and, before an env's last solver stage, the factorisations of the polish's Newton steps
 * in FP32 (the FP64 residuals make the polish an iterative refinement that still reaches the FP64
 * acceptance tolerance; an env's last stage factors in FP64). */

enum { DS_MODE_BREAKING = 0, DS_MODE_STICKING = 1, DS_MODE_SLIDING = 2, DS_MODE_INACTIVE = 3 };

/* per-environment status bits (env_status[e]) */
#define DS_ENV_NOT_CONVERGED 1u  /* the NCP residual check failed after all ADMM stages          */
#define DS_ENV_NONFINITE     2u  /* NaN/Inf in the inputs or the results of this env            */
#define DS_ENV_SINGULAR      4u  /* the reduced implicit system was rank deficient (basic solution used) */
#define DS_ENV_NEAR_SWITCH   8u  /* mode-classification margin below margin_delta               */
#define DS_ENV_BAD_SLOT     16u  /* a contact slot beyond the model's declared slot count is in use */
#define DS_ENV_QUEUE_TIMEOUT 32u  /* persistent launch: not processed, because a wait of the work */
                                  /* queue ran out (queue_poll_limit); v_next holds NaN and the   */
                                  /* env's other outputs are not written                          */

/* Host description of a kinematic tree; copied by ds_model_create (the caller keeps ownership).
 * Bodies are numbered in depth-first preorder (parent[i] < i and every subtree is a contiguous
 * index range).  Body 0 may have a free-flyer joint (joint_type 1); all others are revolute (0). */
typedef struct {
  int32_t nbodies;
  const int32_t* parent;      /* [nbodies], -1 = world                                        */
  const int32_t* joint_type;  /* [nbodies], 0 revolute, 1 free-flyer                           */
  const double* axis;         /* [nbodies][3] unit rotation axis in the joint frame (revolute)   */
  const double* joint_rot;    /* [nbodies][9] row-major rotation of the joint frame in the parent */
  const double* joint_pos;    /* [nbodies][3] origin of the joint frame in the parent            */
  const double* mass;         /* [nbodies]                                                      */
  const double* com;          /* [nbodies][3] centre of mass in the body frame                   */
  const double* inertia;      /* [nbodies][6] (xx, yy, zz, xy, xz, yz) about the centre of mass  */
} ds_model_desc;

typedef struct ds_model ds_model; /* opaque; holds a device copy of the description */

/* Validate and copy a model to the current device.  Errors: DS_EINVAL (bad description),
 * DS_ENOMEM / DS_ECUDA (device copy).  The handle is destroyed with ds_model_destroy.          */
ds_status ds_model_create(const ds_model_desc* desc, ds_model** out);
ds_status ds_model_destroy(ds_model* model);
ds_status ds_model_dims(const ds_model* model, int32_t* nbodies, int32_t* nq, int32_t* nv);

typedef struct {
  int32_t B;                 /* number of environments (>= 0)                                */
  int32_t ncmax;             /* contact slots per environment (0..16)                        */
  const int32_t* model_id;   /* [B] index into the models array, or NULL = every env uses models[0] */
  const double* q;           /* [nq_max][B] */
  const double* v;           /* [nv_max][B] */
  const double* tau;         /* [nv_max][B] */
  const int32_t* c_link;     /* [ncmax][B]  */
  const double* c_point;     /* [ncmax][3][B] */
  const double* c_radius;    /* [ncmax][B]  */
  const double* c_mu;        /* [ncmax][B]  */
  const double* plane;       /* [4][B]      */
  const int32_t* model_slots; /* HOST array [nmodels] or NULL: envs of models[k] use only the
                               * leading model_slots[k] (0..ncmax) slots, the rest hold -1.  Lets a
                               * batch that mixes robots (ncmax set by the one with most contacts)
                               * run every model with a kernel sized for its own contact count;
                               * NULL = ncmax for every model.  A used slot at or beyond the
                               * declared count is ignored and flagged DS_ENV_BAD_SLOT.          */
} ds_batch;

typedef struct {
  double dt;                 /* time step (s) */
  double gravity[3];         /* m/s^2, world frame */
  int32_t admm_max_iter;     /* total ADMM iteration cap per env over all stages               */
  double admm_eps;           /* first (loose) ADMM stage tolerance; later stages tighten it     */
  int32_t polish_iters;      /* Newton steps per stage on the identified mode equations         */
  double ncp_tol;            /* accepted NCP residual, relative to max(1, ||g||_inf)            */
  double eps_sigma;          /* mode test: contact-velocity threshold, relative                */
  double eps_lambda;         /* mode test: impulse threshold, relative                         */
  double margin_delta;       /* DS_ENV_NEAR_SWITCH below this classification margin             */
  int32_t precision;         /* ds_precision */
  double baumgarte_kp;       /* Baumgarte stabilisation (App. D): each active contact's normal   */
  double baumgarte_kd;       /* entry of g gains phi/dt - kp [phi/dt]_- - kd (J_c v)_N, phi its  */
                             /* signed distance ([x]_- = min(x, 0)); the Jacobians and the VJP */
                             /* include the term's derivatives.  kp = 1, kd = 0 (the defaults) */
                             /* add nothing when contact_margin = 0; non-finite gains: DS_EINVAL */
  double contact_margin;     /* activation distance: a slot is active when phi <= contact_margin */
                             /* (>= 0, default 0).  A contact active at phi > 0 gains phi/dt -   */
                             /* kd (J_c v)_N in g (the term above; the proportional part acts  */
                             /* on penetration only), so it may approach the plane by at most   */
                             /* phi within the step.  Negative or non-finite: DS_EINVAL         */
  int32_t ncp_solver;        /* ds_solver (default DS_ADMM); other values: DS_EINVAL             */
  int32_t queue_poll_limit;  /* persistent launch (a schedule of ds_autotune / ds_set_schedule):  */
                             /* polls (~256 ns apart) a CTA makes of the work queue's partition */
                             /* count before it gives up; the envs then left unprocessed get    */
                             /* DS_ENV_QUEUE_TIMEOUT.  Default 2^22; negative: DS_EINVAL         */
  int32_t admm_rho_adapt;    /* 1: adaptive ADMM penalty (an ADMM variant among the solver      */
                             /* alternatives of Sec. 2.2): between the solver's rounds, residual */
                             /* balancing of rho on each env's iterate (primal ||x - z||, dual   */
                             /* ||y + sigma + Gamma(sigma)||; a tenfold imbalance doubles or     */
                             /* halves rho) and K = (G + rho I)^-1 formed again when it changes; */
                             /* same fixed points, same Newton polish and FP64 acceptance.      */
                             /* 0 (default): fixed rho.  ADMM only; other values: DS_EINVAL      */
} ds_options;

/* Fill *opt with the defaults used by the tests and the benchmark (start from these and set the
 * fields to change, so that fields added later keep their defaults). */
void ds_options_default(ds_options* opt);

typedef struct {
  double* v_next;            /* [nv_max][B]  required */
  double* q_next;            /* [nq_max][B]  may be NULL */
  double* lambda;            /* [3*ncmax][B] may be NULL */
  uint8_t* modes;            /* [ncmax][B]   may be NULL */
  uint32_t* env_status;      /* [B]          may be NULL */
  int32_t* iters;            /* [B] ADMM iterations used, may be NULL */
} ds_step_out;

/* Bytes of device workspace that sim_step / sim_step_jac / sim_step_vjp can use for this batch
 * (about 8.1 KB per env for the 7-dof arm with 4 contact slots, 2.4 KB of it the contact
 * problem and the solver state, the rest the forward quantities the setup keeps for the finish,
 * in rows sized also for the split finish's column state; about 45 KB for the 36-dof humanoid
 * with 8).  With a workspace the step runs as a pipeline of
 * kernels (setup, NCP solve in compacted ADMM rounds, finish) that keeps warps busy when the
 * per-env iteration counts differ; without one (workspace = NULL) a single fused kernel does
 * everything.  Both compute the same step; they differ only by rounding (the NCP solve is
 * organised differently across kernels).  The size depends on the models (their forward state)
 * and the batch.  Errors: DS_EINVAL (a NULL model among them, or a model with no compiled kernel for
 * its contact slots). */
ds_status ds_workspace_size(const ds_model* const* models, int32_t nmodels, const ds_batch* batch,
                            const ds_options* opt, size_t* bytes);

/* One step (Eq. 1, 3, 4, 6) for every env.  models[model_id[e]] describes env e; the kernel of a
 * model is the compiled shape (bodies, dofs, slots S) with model_slots[k] <= S <= ncmax and the
 * fewest slots (DS_EUNSUPPORTED if none).  With a workspace and several models, each model's
 * pipeline runs on a helper stream of the library (forked from and joined back to `stream` with
 * events, so the call stays ordered on `stream`); the first such call on a device creates those
 * streams (make it outside stream capture).  Without a workspace the models run one after the
 * other on `stream`.  With a workspace the finish of the envs solved early may also run on a helper
 * stream (the schedule's overlap, see ds_autotune), joined back to `stream` before the call's work
 * ends there.  workspace:
 * NULL, or caller-owned device memory of at least ds_workspace_size() bytes (aligned to 256 bytes),
 * not used concurrently by another call. */
ds_status sim_step(const ds_model* const* models, int32_t nmodels, const ds_batch* batch,
                   const ds_options* opt, const ds_step_out* out, void* workspace,
                   size_t workspace_bytes, void* stream);

/* One step plus the full Jacobians dv+/dq (tangent), dv+/dv, dv+/dtau (Sec. 3, App. D; each
 * [nv][nv][B]).  Envs of different models must all have nv equal to the row count of the arrays:
 * element (i, j) of env e is at (i*nv_e + j)*B + e with nv_e the env's own nv. */
ds_status sim_step_jac(const ds_model* const* models, int32_t nmodels, const ds_batch* batch,
                       const ds_options* opt, const ds_step_out* out, double* dv_dq, double* dv_dv,
                       double* dv_dtau, void* workspace, size_t workspace_bytes, void* stream);

/* Vector-Jacobian product (reverse mode, the OptNet-style adjoint of Sec. 3.1): given
 * v_next_bar [nv_max][B], writes q_bar (tangent), v_bar, tau_bar [nv_max][B] =
 * (dv+/d(q, v, tau))^T v_next_bar without forming the Jacobians.  Also fills *out like sim_step.
 * q_next_bar [nv_max][B] (may be NULL): a cotangent of q+ as well, in the tangent coordinates at
 * q+ (the free-flyer's (linear, angular) in its own frame).  The adjoint of the position update
 * q+ = q (+) dt v+ (symplectic Euler, Sec. 2.3) is then chained in: the step's outputs get the
 * cotangent of (q+, v+) jointly, which is what a rollout's backward pass passes from step to step. */
ds_status sim_step_vjp(const ds_model* const* models, int32_t nmodels, const ds_batch* batch,
                       const ds_options* opt, const double* v_next_bar, const double* q_next_bar,
                       const ds_step_out* out, double* q_bar, double* v_bar, double* tau_bar,
                       void* workspace, size_t workspace_bytes, void* stream);

/* sim_step_vjp from a tape: the same VJP, for the solution a preceding sim_step (or sim_step_jac /
 * sim_step_vjp) on the same inputs and options returned, without solving the NCP again.  tape:
 * that call's outputs lambda [3*ncmax][B], modes [ncmax][B] and env_status [B] (required; other
 * fields ignored).  Only the finish kernel runs (kinematics, dynamics and contact Jacobians are
 * recomputed from the inputs; lambda and the modes come from the tape), so a rollout's reverse pass
 * differentiates exactly the trajectory its forward pass produced.  No workspace.  *out is filled
 * like sim_step's (v_next required).  Errors: DS_EINVAL (missing tape arrays, as sim_step_vjp),
 * DS_EUNSUPPORTED, DS_ECUDA. */
ds_status sim_step_vjp_tape(const ds_model* const* models, int32_t nmodels, const ds_batch* batch,
                            const ds_options* opt, const double* v_next_bar, const double* q_next_bar,
                            const ds_step_out* tape, const ds_step_out* out, double* q_bar, double* v_bar,
                            double* tau_bar, void* stream);

const char* ds_status_string(ds_status s);

/* Cotangent coordinate maps for the configuration (the derivative convention above: q (+) eta with
 * position += R eta_lin and quaternion <- quaternion * exp(eta_ang / 2), Sec. 2.3's integrator on
 * the configuration manifold).  Callers whose losses are written in the raw coordinates of q
 * (nq numbers per env, quaternion included) use them at the two ends of a reverse pass:
 *   ds_cotangent_to_tangent: q_bar_tangent [nv_max][B] = (dq_raw/deta)^T q_bar_raw [nq_max][B];
 *   ds_cotangent_to_raw:     q_bar_raw [nq_max][B] = (deta/dq_raw)^T q_bar_tangent [nv_max][B],
 *                            which has no component along the quaternion (normalisation).
 * q [nq_max][B] is the configuration at which the cotangents live; model_id as in ds_batch (NULL
 * when nmodels == 1).  Revolute rows are copied.  Asynchronous on stream; errors: DS_EINVAL, DS_ECUDA. */
ds_status ds_cotangent_to_tangent(const ds_model* const* models, int32_t nmodels, int32_t B,
                                  const int32_t* model_id, const double* q, const double* q_bar_raw,
                                  double* q_bar_tangent, void* stream);
ds_status ds_cotangent_to_raw(const ds_model* const* models, int32_t nmodels, int32_t B,
                              const int32_t* model_id, const double* q, const double* q_bar_tangent,
                              double* q_bar_raw, void* stream);

/* Allocation-free sim_step_jac (no counterpart in the paper; a convenience of this library).
 * Some callers cannot allocate device memory when they step the simulation: a real-time control
 * loop that forbids allocation after start-up (allocation latency is unbounded), or a plug-in that
 * does not own the process's CUDA memory.  This call computes exactly what sim_step_jac computes
 * with a workspace, but takes that workspace from a fixed array of DS_NOALLOC_SCRATCH_BYTES
 * (16 MiB) that the library holds on every device that loads it, until the process exits.  It
 * calls no cudaMalloc / cudaFree and no allocating routine.
 *   - Batches whose ds_workspace_size() exceeds the array are rejected with DS_ETOOLARGE
 *     (about 2070 envs of the 7-dof arm with 4 contact slots).
 *   - The first call on a device resolves the array's device address (cudaGetSymbolAddress);
 *     make that first call outside any stream capture.
 *   - Every call shares the one array and leaves its contents behind; the counters that must
 *     start at zero are cleared by each call.  Calls whose work overlaps on the GPU (different
 *     streams, or host threads without ordering) race on the array: serialize them.
 * Arguments, outputs and errors otherwise as for sim_step_jac. */
#define DS_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
ds_status sim_step_jac_noalloc(const ds_model* const* models, int32_t nmodels, const ds_batch* batch,
                               const ds_options* opt, const ds_step_out* out, double* dv_dq, double* dv_dv,
                               double* dv_dtau, void* stream);

/* Schedule autotuning (no counterpart in the paper).  How the workspace pipeline divides its work
 * is a schedule: the table of ADMM round caps (how many iterations an env may run before the
 * lists are compacted: default {32, 32, 64, ..., 4096}, halved, or doubled; the last round always
 * runs to the iteration limit), the first round handled by the row-per-lane ADMM kernel (3, 5 or
 * never), how many threads share an env's Jacobian columns in the finish kernel (a target of 0, 4
 * or 8 CTAs per SM), the Newton kernel's form (cooperative or one thread per env), and the round
 * after which the envs already solved are finished on a side stream of the library while the slow
 * ones still iterate (right after the setup, 2, 4, 5 or never), the first round handled by the
 * two-warp ADMM kernel (FP64 with at most 10 contact slots: one warp runs the x-step and
 * projection, the other the De Saxce term and convergence test; 3, 5 or never), and which SMs that overlapped finish leaves to
 * the slow envs (none, every 8th or every 4th: the FP64 pipe of an SM sub-partition is shared by
 * its warps, so the late rounds run faster on SMs the finish does not occupy), and the round from
 * whose end on the Newton / active-set stage also tries the iterate of every env still iterating,
 * not only of those whose ADMM stage tolerance was met, with a fallback that enumerates the
 * contact-mode patterns with one or two contacts in contact when the active-set rounds fail
 * (speculative attempts from round 3, from round 5, or never; an env whose attempt fails keeps
 * iterating in the same stage), and whether the setup solves Eq. 1 exactly for the envs whose
 * solution has a single contact in contact and every other contact breaking (the sticking
 * impulse -G_ii^-1 g_i, else Newton on the sliding equations from its cone projection, accepted by
 * the same FP64 NCP residual test as the Newton stage), so that those envs skip the ADMM rounds;
 * and whether the step runs as the pipeline above or as one persistent launch: a kernel sized to
 * the CTAs the GPU keeps resident, whose warps pull chunks of 32 envs of one model from an atomic
 * work queue (the costliest model's chunks first) and run one env per lane through the whole
 * step (the fused per-env form of every stage), all models of the batch in the same kernel.  The
 * persistent launch exists for the shapes compiled into it (a 7-dof arm with 8 contact slots, an
 * 18-dof quadruped with 4 and a 36-dof humanoid with 16, DS_MIXED only) and at most 4
 * models; a batch with another shape runs the pipeline under such a schedule.  Its queue can
 * only be read once every CTA has filed its share of the envs into the per-model lists; a CTA
 * polls for that at most queue_poll_limit times (ds_options), and when one gives up, every CTA
 * stops claiming work and the envs left get DS_ENV_QUEUE_TIMEOUT.  And the finish's form: one
 * kernel whose threads each hold an env (or a share of its columns) in registers and local
 * memory, or two: a prep kernel, one thread per env, that does the step's outputs, the reduced
 * implicit system and its factor and the rows of the implicit part (Jacobians) or the adjoint
 * vectors (VJP), and stores what the columns read in the workspace; then a column kernel, one
 * warp per env, that stages that state in shared memory and spreads the 3 nv Jacobian columns
 * (the VJP's 2 nv dof passes) over its lanes (in the mixed form the implicit part is then applied
 * in FP32 instead of FP64).
 * ds_autotune runs `mode` (0 = sim_step, 1 = sim_step_jac with o0..o2 = dv_dq, dv_dv, dv_dtau,
 * 2 = sim_step_vjp with v_next_bar and o0..o2 = q_bar, v_bar, tau_bar) on this batch, timing each
 * schedule by the second slowest of five runs (so that a schedule whose step time varies from
 * run to run is judged by its slow runs; CUDA events on `stream`, after an untimed run; before each
 * run the call writes a 256 MB scratch buffer of its own, allocated and freed by the call, so that
 * every run starts with a cold L2 as a step of a real loop does), in a
 * coordinate search from the default (each knob over its options with the others at the best so
 * far, two passes over the knobs; a schedule replaces the best only if 2 % faster).  It keeps the
 * fastest for the batch's signature (first model's bodies and dofs, number of models, ncmax,
 * precision, mode, B rounded up to a power of two) and finally runs the call once more with it,
 * so that *out and o0..o2 hold its results.  Later calls with the same signature use that
 * schedule; other batches keep the default.  A schedule changes how the work is divided, and what
 * an env computes only within the solver tolerance: the two Newton forms round differently, so
 * does the two-warp ADMM kernel's x-step (summed in two halves) for models of 2 or 4 contact
 * slots, and the round caps and speculative attempts decide at which iterates the Newton stage
 * runs (every accepted impulse passes the same NCP residual test; where Eq. 1 has several
 * solutions, two schedules can return different ones).
 * Blocking: it synchronises on `stream`.  The workspace is required.  *chosen (may be NULL) gets
 * the schedule's index (0 .. 58319), the mixed-radix number c + 3 (w + 3 (f + 3 (n + 2 (o + 5 (p +
 * 3 (r + 3 (s + 3 (x + 2 (u + 2 h))))))))): round caps c (0 default, 1 halved, 2 doubled), first row-per-lane
 * round w (0: 3, 1: 5, 2: never), finish target f (0, 4, 8 CTAs per SM as 0, 1, 2), Newton n (0
 * cooperative, 1 one thread per env), overlapped finish o (0: after the setup, 1: after round 2,
 * 2: after round 4, 3: after round 5, 4: never), two-warp ADMM p (0: from round 3, 1: from round 5,
 * 2: never), SMs kept
 * free r (0: none, 1: every 8th, 2: every 4th), speculative Newton attempts s (0: from round 3, 1:
 * from round 5, 2: never), single-contact presolve x (0 on, 1 off), launch u (0 pipeline, 1
 * persistent), finish h (0 one kernel, 1 prep + column kernels).  Errors: DS_EINVAL, DS_ECUDA,
 * those of the call. */
ds_status ds_autotune(const ds_model* const* models, int32_t nmodels, const ds_batch* batch,
                      const ds_options* opt, int32_t mode, const double* v_next_bar, const ds_step_out* out,
                      double* o0, double* o1, double* o2, void* workspace, size_t workspace_bytes,
                      void* stream, int32_t* chosen);

/* Sets the schedule (index as ds_autotune's *chosen) that later calls of `mode` use for batches
 * with this batch's signature, as if ds_autotune had chosen it; index -1 returns the signature to
 * the default schedule (no counterpart in the paper).  For reusing a tuned schedule without timing
 * again, and for running a given kernel form.  Errors: DS_EINVAL (index outside -1 .. 58319). */
ds_status ds_set_schedule(const ds_model* const* models, int32_t nmodels, const ds_batch* batch,
                          const ds_options* opt, int32_t mode, int32_t index);

/* Checked build (no counterpart in the paper; a debugging aid, libdiffsim_check.so, built with
 * -DDS_CHECK).  There every tree index (bodies, parents, dofs, subtrees), every env index read
 * from the pipeline's work lists and every shared-memory group index of the Newton kernel is
 * checked against its range; an index out of range is counted and replaced by 0, so that it shows
 * up as a count instead of a memory fault.  ds_check_bad_indices synchronises the device, writes
 * the count summed over the kernels since the last call to *count and clears it.
 * ds_check_self_test launches one check of `index` against [0, n) and writes the count it gives
 * (1 for an index outside the range, 0 inside): the counting itself, tested.  In the normal build
 * both return DS_EUNSUPPORTED with *count = 0.  Errors: DS_EINVAL (NULL count, n <= 0), DS_ECUDA. */
ds_status ds_check_bad_indices(uint64_t* count);
ds_status ds_check_self_test(int32_t index, int32_t n, uint64_t* count);

/* Stage tracing (no counterpart in the paper): with ds_profile(1), every kernel the library
 * launches is bracketed by CUDA events on its own stream, grouped in DS_NSTAGES = 5 classes:
 * 0 setup, 1 ADMM rounds, 2 Newton / active-set, 3 finish (step update + derivatives), 4 fused
 * single-kernel path.  ds_profile_read waits for the recorded events, writes the summed
 * milliseconds and launch counts per class to ms[5], launches[5], and clears the record (kernels
 * of different models that overlap in time are each counted in full). */
ds_status ds_profile(int32_t enable);
ds_status ds_profile_read(double* ms, int32_t* launches);

/* ---------------------------------------------------------------------------------------------
 * Collision detection between convex shapes (Sec. 2.1; App. C writes it as the contact placement
 * 0M_c = CD(0M_1, 0M_2)).  Not yet used by the step, whose contacts are primitive-versus-plane.
 *
 * A shape is a type and three sizes: DS_CONVEX_SPHERE (radius, -, -), DS_CONVEX_CAPSULE (half
 * length, radius, -; the segment runs along the body z axis from -half length to +half length),
 * DS_CONVEX_BOX (half extents hx, hy, hz), DS_CONVEX_HULL (first vertex, vertex count, radius: the
 * convex hull of vertices first .. first + count - 1 of the pool hull_vertices, in the body frame,
 * swept by the radius; 4 <= count <= DS_CONVEX_HULL_MAX, both integral).  A pose is 12 numbers:
 * the rotation R (row-major, body to world) and the position p.  For each of n_pairs pairs (A, B) ds_collide writes DS_COLLIDE_OUT
 * numbers to out[DS_COLLIDE_OUT * k ...]: the signed distance phi (< 0: penetration), the contact
 * point c[3] (the midpoint of the witness points), the unit normal n[3] from A to B, the tangent
 * axes t1[3], t2[3] of the contact frame (Z along n; t1 = normalize(e_x - (n.e_x) n), e_y in place
 * of e_x when |n_x| > 0.9; t2 = n x t1) and the witness points on A's and B's surfaces sa[3],
 * sb[3].  Separated shapes take the closest points of their cores (point, segment, box corners or
 * hull vertices) by GJK; overlapping ones the penetration depth of the cores along the nearest
 * facet of their Minkowski difference (separating axes for a box with a point, segment or box;
 * the expanding polytope, EPA, with a hull).  Touching or crossing point and segment cores (sphere and capsule cores)
 * have no normal: n is the world z axis there.  Where the witness points are not unique (parallel
 * faces or edges in contact) one of them is returned.
 *
 * Pointers: type_a, type_b (int32, n_pairs), size_a, size_b (FP64, 3 n_pairs), pose_a, pose_b
 * (FP64, 12 n_pairs) and out (FP64, DS_COLLIDE_OUT n_pairs) are device pointers, read and written
 * on `stream` (a cudaStream_t, NULL = the default stream); the call returns after the launch.
 * The caller owns every buffer.  Errors: DS_EINVAL (n_pairs < 0, or a NULL pointer with
 * n_pairs > 0), DS_ECUDA (launch failure).  A pair with an unknown type gets NaN in all its
 * outputs, and so does a hull whose range is not inside the pool or a hull penetration that the
 * expanding polytope cannot resolve within 64 vertices and 128 faces.  hull_vertices (FP64,
 * 3 n_hull_vertices, device) may be NULL when no pair has a hull.  n_pairs = 0 launches nothing. */
enum { DS_CONVEX_SPHERE = 0, DS_CONVEX_CAPSULE = 1, DS_CONVEX_BOX = 2, DS_CONVEX_HULL = 3 };
#define DS_COLLIDE_OUT 19
#define DS_CONVEX_HULL_MAX 32
ds_status ds_collide(int32_t n_pairs, const int32_t* type_a, const double* size_a, const double* pose_a,
                     const int32_t* type_b, const double* size_b, const double* pose_b,
                     const double* hull_vertices, int32_t n_hull_vertices, double* out, void* stream);

/* The derivative App. C takes of the collision detection: its zero-order randomized-smoothing
 * estimate.  For each pair, with the caller's samples eps_s = (u_A, w_A, u_B, w_B) (s < n_samples,
 * 12 numbers each, drawn from N(0, sigma^2 I); the same samples serve every pair), the poses are
 * moved by +-eps_s as world-frame twists (x -> exp([w]) x + V(w) u: R' = exp([w]) R,
 * p' = exp([w]) p + V(w) u) and
 *   J = 1 / (2 n_samples sigma^2) sum_s (f(+eps_s) - f(-eps_s)) eps_s^T,
 * f = (phi, c[3], n[3]) the first 7 outputs of ds_collide.  J is the gradient estimate of the
 * Gaussian-smoothed f with respect to the two twists: 7 x 12, row-major (columns: A's u, A's w,
 * B's u, B's w), written to jac[84 k ...].  Shapes, poses and hulls as for ds_collide; eps (FP64,
 * 12 n_samples) and jac (FP64, 84 n_pairs) are device pointers.  Errors: DS_EINVAL (n_pairs < 0,
 * n_samples <= 0 with n_pairs > 0, sigma not positive and finite, a NULL pointer with
 * n_pairs > 0), DS_ECUDA (launch failure). */
ds_status ds_collide_smoothed(int32_t n_pairs, const int32_t* type_a, const double* size_a, const double* pose_a,
                              const int32_t* type_b, const double* size_b, const double* pose_b,
                              const double* hull_vertices, int32_t n_hull_vertices, int32_t n_samples,
                              const double* eps, double sigma, double* jac, void* stream);

/* Measurement helper (no counterpart in the paper): runs `blocks` x 256 threads, each doing `iters`
 * rounds of 8 independent fused multiply-adds in FP64 (fp64 != 0) or FP32 and writing one value per
 * thread to out[blocks*256] (device, FP64).  Used to measure the CUDA-core FMA peak that bounds
 * this ALU-bound path; 2 * 8 * iters * blocks * 256 flops per launch. */
ds_status ds_fma_peak(double* out, int32_t blocks, int32_t iters, int32_t fp64, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* DIFFSIM_H */
