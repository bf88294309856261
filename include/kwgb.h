/*
 * kwgb.h -- C ABI of the GB300 k-space pseudospectral time step.
 *
 * The library advances the coupled first-order acoustic equations of
 * Jaros, Rendell & Treeby, "Full-wave nonlinear ultrasound simulation on
 * distributed clusters with applications in HIFU" (Sec. 2, Eqs. 1-8) on one
 * GPU: 3D real-to-complex / complex-to-real FFTs, the kappa k-space
 * correction and staggered-grid shift operators (Eqs. 4a, 4c), the split-field
 * PML velocity and density updates (Eqs. 4b, 4d), the power-law absorption
 * term (Eq. 8) and the nonlinear equation of state (Eq. 6).
 *
 * Conventions
 *  - Grid arrays are float32, C order [nz][ny][nx] (x fastest); the linear
 *    index of (x, y, z) is x + nx * (y + ny * z).
 *  - u_xi is stored at the staggered point x_i + dxi/2 (Sec. 2.2, Fig. 1).
 *  - Every input array is COPIED by the library; the caller keeps ownership.
 *    Input pointers are host pointers unless the call says otherwise.
 *  - Functions return KWGB_OK (0) or a negative KWGB_ERR_* code; the message
 *    of the last failure on a simulation is returned by kwgb_last_error().
 *    Nothing traps or aborts on the device; device-side problems (non-finite
 *    pressure) raise a flag that the next synchronising call reports.
 *  - kwgb_step() is asynchronous on the caller's CUDA stream; kwgb_read(),
 *    kwgb_read_field() and kwgb_status() synchronise with it.
 *  - Supported grids: nx, ny, nz powers of two in [8, 1024] (the FFT passes
 *    are radix-2^k shared-memory kernels); anything else is KWGB_ERR_UNSUPPORTED.
 *  - Calls on one simulation are not thread safe; separate simulations are
 *    independent.
 */
#ifndef KWGB_H
#define KWGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------ */
#define KWGB_OK                0
#define KWGB_ERR_ARG          -1  /* invalid argument (null, size, range)      */
#define KWGB_ERR_OOM          -2  /* device allocation failed                  */
#define KWGB_ERR_CUDA         -3  /* a CUDA runtime call failed                */
#define KWGB_ERR_NONFINITE    -4  /* pressure became NaN/Inf during stepping   */
#define KWGB_ERR_TIMEOUT      -5  /* a bounded device wait ran out             */
#define KWGB_ERR_STATE        -6  /* call not allowed in the current state     */
#define KWGB_ERR_UNSUPPORTED  -7  /* valid request the library does not serve  */

/* ---- grid flags (kwgb_grid_desc.flags) ---------------------------------- */
#define KWGB_NONLINEAR   1u  /* Eq. 4d denominator and (B/2A) rho^2/rho0 of Eq. 6 */
#define KWGB_ABSORBING   2u  /* power-law absorption/dispersion L_d of Eq. 8     */
#define KWGB_MIXED_BF16  4u  /* y/z FFTs as bfloat16-split tensor-core products with float32 accumulation
                                (tcgen05 radix-32 stages for lines of 64 points and more, mma.sync radix-8
                                for 16- and 32-point lines); needs ny, nz >= 16 */
#define KWGB_MIXED_F16   8u  /* same with float16 hi + lo and a per-column power-of-two scale; needs ny, nz >= 16 */

/* ---- sensor outputs (kwgb_add_sensor record / kwgb_read which) ---------- */
#define KWGB_P_MAX  1u   /* max_n p^n, n = 1..Nt                               */
#define KWGB_P_RMS  2u   /* sqrt(mean_n (p^n)^2)                               */
#define KWGB_I_AVG  4u   /* time-averaged intensity, 3 components per point    */
#define KWGB_P_MIN  8u   /* min_n p^n (peak negative pressure)                 */
#define KWGB_P_SERIES 16u /* p^n at every step (ring of the last `capacity`    */
                          /* steps, see kwgb_set_series_capacity)              */
#define KWGB_U_SERIES 32u /* u_x, u_y, u_z^{n-1/2} at every step (same ring;   */
                          /* the value at the staggered point, no averaging)   */

/* ---- source modes ------------------------------------------------------- */
#define KWGB_ADDITIVE_MASS 0  /* mass source M of Eq. 4d, see kwgb_add_source  */
#define KWGB_FORCE_X 1        /* force density along x, see kwgb_add_source    */
#define KWGB_FORCE_Y 2
#define KWGB_FORCE_Z 3
#define KWGB_DIRICHLET_P 4    /* pressure held at the signal, see kwgb_add_source */

/* ---- objectives of kwgb_adjoint ----------------------------------------- */
#define KWGB_OBJ_MEAN_ABS_P 0  /* J = 1/(n_obj Nt) sum_{n=1..Nt} sum_i |p^n(idx_i)| */

/* ---- kwgb_set_medium scalar_mask bits ----------------------------------- */
#define KWGB_SCALAR_C0      1u
#define KWGB_SCALAR_RHO0    2u
#define KWGB_SCALAR_BONA    4u
#define KWGB_SCALAR_ALPHA0  8u
#define KWGB_INPUT_DEVICE   0x80000000u /* non-scalar arrays are device pointers */

/* ---- fields for kwgb_read_field ----------------------------------------- */
#define KWGB_FIELD_P     0   /* p^n                  */
#define KWGB_FIELD_UX    1   /* u_x^{n-1/2}          */
#define KWGB_FIELD_UY    2
#define KWGB_FIELD_UZ    3
#define KWGB_FIELD_RHOX  4   /* rho_x^n (split field) */
#define KWGB_FIELD_RHOY  5
#define KWGB_FIELD_RHOZ  6

/* ---- spectral operators for kwgb_apply_operator ------------------------- */
#define KWGB_OP_GRAD_FWD 0   /* Eq. 4a: IFT{ i k_xi kappa e^{+i k_xi dxi/2} FT{f} }, 3 outputs */
#define KWGB_OP_GRAD_BWD 1   /* Eq. 4c: IFT{ i k_xi kappa e^{-i k_xi dxi/2} FT{f} }, 3 outputs */
#define KWGB_OP_ABS_TAU  2   /* Eq. 8:  IFT{ k^{y-2} FT{f} }, 1 output (0 at k = 0)           */
#define KWGB_OP_ABS_ETA  3   /* Eq. 8:  IFT{ k^{y-1} FT{f} }, 1 output (0 at k = 0)           */

typedef struct kwgb_sim kwgb_sim;  /* opaque; owned by the library */

/* Grid and run parameters (Sec. 2.2; Eq. 5 wavenumbers).
 *   nx, ny, nz    grid points (powers of two, 8..1024)
 *   dx, dy, dz    spacing [m];  dt  time step [s]
 *   c_ref         reference sound speed of kappa = sinc(c_ref k dt/2) [m/s]
 *   pml_size      PML thickness in cells per axis (0 = none), inside the grid
 *   pml_alpha     PML strength per axis [Np per grid point]; the absorption is
 *                 alpha * (c_ref/dxi) * (depth/size)^4, depth measured in cells
 *                 from the inner edge of the layer
 *   flags         KWGB_NONLINEAR | KWGB_ABSORBING, optionally one of KWGB_MIXED_BF16 / KWGB_MIXED_F16
 *   alpha_power   power-law exponent y (Eq. 3), 0 < y < 3, y != 1; one value
 *                 for the whole grid                                          */
typedef struct {
    int64_t nx, ny, nz;
    double dx, dy, dz, dt, c_ref;
    int32_t pml_size[3];
    double pml_alpha[3];
    uint32_t flags;
    double alpha_power;
} kwgb_grid_desc;

/* Validate desc and create an empty simulation.  No device memory is taken
 * until kwgb_set_medium().  *out receives the handle (NULL on failure).
 * Errors: ARG (null, non-positive spacing or dt, PML too thick, y outside
 * (0,3) or y == 1 when absorbing), UNSUPPORTED (sizes). */
int kwgb_create(const kwgb_grid_desc* desc, kwgb_sim** out);

/* Route the simulation's device allocations through alloc/free (for example
 * a framework's caching allocator).  alloc(bytes, ctx) returns a device
 * pointer aligned to 256 bytes or NULL; free(ptr, ctx) releases it.  Must be
 * called before kwgb_set_medium().  Errors: ARG, STATE. */
int kwgb_set_allocator(kwgb_sim* sim, void* (*alloc)(size_t bytes, void* ctx),
                       void (*free_fn)(void* ptr, void* ctx), void* ctx);

/* Medium (Eq. 1/3): sound speed c0 [m/s], ambient density rho0 [kg/m^3],
 * nonlinearity B/A, and the power-law prefactor alpha0 in
 * Np (rad/s)^-y m^-1.  Each pointer refers to nx*ny*nz floats, or to one
 * float when its KWGB_SCALAR_* bit is set in scalar_mask; b_on_a and alpha0
 * may be NULL (= 0).  With KWGB_INPUT_DEVICE set, the non-scalar arrays are
 * device pointers (scalars are always host).  Allocates all device state
 * and zeroes p, u, rho.  Errors: ARG, OOM, CUDA, STATE (already set). */
int kwgb_set_medium(kwgb_sim* sim, const float* c0, const float* rho0,
                    const float* b_on_a, const float* alpha0, uint32_t scalar_mask);

/* Initial pressure p0 (host, nx*ny*nz floats).  Sets p^0 = p0,
 * rho_xi^0 = p0/(3 c0^2) and u_xi^{-1/2} = +dt/(2 rho0_sg) d/dxi p0 (Eq. 4a
 * operator), so that the velocity is zero at t = 0.  Before the first step
 * only.  Errors: ARG, STATE, CUDA. */
int kwgb_set_initial_pressure(kwgb_sim* sim, const float* p0);

/* Additive mass source (the M term of Eq. 4d) at n_idx linear indices idx
 * (host int64, each in [0, nx*ny*nz)).  signal (host) holds n_signals rows
 * of n_t samples: n_signals == 1 drives every point with the same signal,
 * n_signals == n_idx gives point i its own row.  Sample n drives time step n
 * (t = (n + 1/2) dt); after n_t steps the source is silent.  At each point
 * every split density gets rho_xi += dt * 2 s / (3 c0 dx), so a planar source
 * radiates a plane wave of amplitude s.  Points may repeat and sources may
 * overlap (contributions add).  Before the first step only.
 * mode KWGB_FORCE_X / _Y / _Z instead adds a force density F [N/m^3] along
 * that axis (the paper's velocity-updating source kind, Sec. 3.4): after the
 * velocity update of Eq. 4b, u_xi += dt F / rho0_sg at the staggered point of
 * each index, sample n at t = n dt; a planar force layer radiates pressure
 * +-F dxi/2 on its two sides.
 * mode KWGB_DIRICHLET_P sets the pressure at the points (Sec. 3.4: a source
 * updates the value of the pressure at its grid points): in step n, after the
 * density update of Eq. 4d and the additive sources, every split density at
 * the point becomes s / (3 c0^2), and after Eq. 6 the pressure p^{n+1}
 * becomes s (sample n; sources sharing a point add); a point is held only in
 * steps for which one of its signals has a sample.  A plane held this way
 * radiates plane waves of amplitude s to both sides.
 * *source_id receives the source number.  Errors: ARG (bad mode, sizes,
 * indices), STATE, OOM, CUDA. */
int kwgb_add_source(kwgb_sim* sim, const int64_t* idx, int64_t n_idx,
                    const float* signal, int64_t n_signals, int64_t n_t,
                    int mode, int32_t* source_id);

/* Sensor at n_idx linear indices idx (host int64), or at every grid point
 * when idx is NULL (then n_idx is ignored).  record is a set of KWGB_P_MAX,
 * KWGB_P_RMS, KWGB_I_AVG, KWGB_P_MIN, KWGB_P_SERIES, KWGB_U_SERIES (the
 * aggregate and time-varying outputs collected at the sensor mask, Sec. 3.4).
 * Samples are p^1 .. p^Nt and u^{1/2} .. u^{Nt-1/2}.  Before the first step
 * only.  A sensor with a series needs kwgb_set_series_capacity before the
 * first step.  *sensor_id receives the sensor number.  Errors: ARG, STATE,
 * OOM. */
int kwgb_add_sensor(kwgb_sim* sim, const int64_t* idx, int64_t n_idx,
                    uint32_t record, int32_t* sensor_id);

/* Length n_t > 0 of the device ring buffer of a series sensor: it keeps the
 * samples of the last n_t steps (n_t >= the run's steps keeps them all).
 * Device memory: 4 n_t n_idx bytes for KWGB_P_SERIES, 12 n_t n_idx for
 * KWGB_U_SERIES.  Before the first step only.  Errors: ARG, STATE. */
int kwgb_set_series_capacity(kwgb_sim* sim, int32_t sensor_id, int64_t n_t);

/* Advance n_steps time steps, (u^{n-1/2}, rho^n, p^n) -> (u^{n+1/2},
 * rho^{n+1}, p^{n+1}) per step, asynchronously on cuda_stream (a
 * cudaStream_t; NULL = the legacy default stream).  n_steps == 0 is a no-op.
 * The first call builds the device lists of the sources and sensors (the
 * indices grouped by grid row on the host, uploaded, one device
 * synchronisation); from then on sources and sensors are fixed.
 * The first step of a simulation launches its kernels directly and the
 * library then captures one step into a CUDA graph (on a stream of its own)
 * that later steps replay on cuda_stream; if capture is not possible the
 * kernels keep being launched directly.  Either way the results are the
 * same.  Errors: ARG (n_steps < 0), STATE (no medium), CUDA. */
int kwgb_step(kwgb_sim* sim, int64_t n_steps, void* cuda_stream);

/* Copy one sensor output to host_out as float64.  which is ONE of
 * KWGB_P_MAX, KWGB_P_MIN, KWGB_P_RMS (n_idx values each), KWGB_I_AVG
 * (3*n_idx values: all x components, then y, then z), KWGB_P_SERIES
 * (m*n_idx values, [sample][point]) or KWGB_U_SERIES (m*3*n_idx values,
 * [sample][component][point]), where m = min(steps taken, capacity) and the
 * series hold the last m samples, oldest first.  n is the capacity of
 * host_out in doubles.  Synchronises.  The intensity's last term needs
 * u^{Nt+1/2}; it is computed here by one extra velocity update that changes
 * no state.  With no step taken p_max = -inf, p_min = +inf, p_rms = 0,
 * I = 0 and the series are empty.
 * Errors: ARG (bad id/which, n too small, output not recorded), CUDA,
 * NONFINITE (pressure went non-finite; the values are still copied). */
int kwgb_read(kwgb_sim* sim, int32_t sensor_id, uint32_t which,
              double* host_out, int64_t n);

/* Copy a state field (KWGB_FIELD_*) at the current step to host_out
 * (nx*ny*nz floats).  Synchronises.  Errors: ARG, STATE, CUDA, NONFINITE. */
int kwgb_read_field(kwgb_sim* sim, int field, float* host_out, int64_t n);

/* Apply one of the step's spectral operators (KWGB_OP_*) to the device field
 * in (nx*ny*nz floats) and write the result(s) to the device arrays out0..2
 * (out1/out2 only for the gradient operators), on cuda_stream, using the
 * simulation's grid and scratch spectra.  The state is not touched.  Needs
 * kwgb_set_medium() first.  Errors: ARG, STATE, CUDA. */
int kwgb_apply_operator(kwgb_sim* sim, int op, const float* in, float* out0,
                        float* out1, float* out2, void* cuda_stream);

/* Allocation-free form of the staggered gradient that kwgb_apply_operator
 * computes for KWGB_OP_GRAD_FWD / KWGB_OP_GRAD_BWD (the paper has no
 * counterpart: it is an interface for callers that cannot allocate device
 * memory, such as code whose device memory is owned entirely by another
 * allocator or a fixed arena, and code that must not allocate after start-up,
 * where cudaMalloc may synchronise the device or fail).
 *   desc      grid: nx, ny, nz powers of two in [8, 64]; dx, dy, dz, dt, c_ref
 *             positive and finite (pml_*, flags and alpha_power are ignored);
 *             no simulation needed
 *   op        KWGB_OP_GRAD_FWD (the spectral gradient shifted half a cell
 *             forward, as the velocity update uses it) or KWGB_OP_GRAD_BWD
 *             (shifted half a cell back, as the density update uses it)
 *   in        device field, nx*ny*nz floats, [nz][ny][nx]
 *   out_x/y/z device outputs, nx*ny*nz floats each (not aliasing in)
 *   err       optional buffer (errlen bytes) that receives a message on failure
 * Asynchronous on cuda_stream.  It allocates nothing and calls no cudaMalloc
 * or cudaFree: its scratch (three spectra and small tables) is one file-scope
 * device array of about 4.7 MB that every GPU loading the library's device
 * code holds until the process exits.  Larger grids are rejected with
 * KWGB_ERR_UNSUPPORTED.
 * The first call on a device does the set-up: under CUDA's lazy module
 * loading it loads the library's device code (which reserves the array),
 * looks up the array's device address (cudaGetSymbolAddress) and uploads the
 * twiddle table, synchronising the device; make it at start-up, before any
 * stream capture.  Later calls enqueue kernels and one memset on cuda_stream
 * and copy nothing from the host.
 * All calls share the array and it keeps the previous call's contents (each
 * call clears its status word and overwrites everything else it reads), so
 * calls that overlap on the GPU, e.g. from two streams, race and must be
 * serialised by the caller.  A device-side failure (a bounded wait that ran
 * out) is not seen by this call: kwgb_gradient_static_status reports it.
 * Errors: ARG, UNSUPPORTED, CUDA. */
int kwgb_gradient_static(const kwgb_grid_desc* desc, int op, const float* in, float* out_x,
                         float* out_y, float* out_z, void* cuda_stream, char* err,
                         size_t errlen);

/* Device status of the kwgb_gradient_static calls on the current device since
 * the last one began: synchronises cuda_stream (the stream of those calls),
 * then reads the shared status word (a synchronous 4-byte copy into the
 * caller's stack; nothing is allocated).  Returns KWGB_OK, KWGB_ERR_TIMEOUT
 * (a bounded tile-load wait ran out; the outputs were not written),
 * KWGB_ERR_NONFINITE, KWGB_ERR_STATE (no call on this device yet) or
 * KWGB_ERR_CUDA; err as for kwgb_gradient_static. */
int kwgb_gradient_static_status(void* cuda_stream, char* err, size_t errlen);

/* Test hook of the failure path of kwgb_gradient_static (the counterpart of
 * kwgb_debug_wait_fault): while on != 0, every tile load of later calls
 * expects 16 bytes more than it receives, so the kernels' bounded waits run
 * out (about 2 s each) and kwgb_gradient_static_status returns
 * KWGB_ERR_TIMEOUT.  No fault is raised and the context stays usable.
 * Returns KWGB_OK. */
int kwgb_gradient_static_debug_wait_fault(int on);

/* Gradient of an objective of the pressure with respect to every source
 * signal sample, by a hand-written adjoint (reverse-mode) of the time step
 * (Eqs. 4a-4d, 6 and 8 run backwards: the transpose of the Eq. 4a operator
 * is minus the Eq. 4c operator and vice versa; the k^{y-2} and k^{y-1}
 * operators of Eq. 8 are real and even, hence their own transposes; Eq. 4d
 * and Eq. 6 by their pointwise derivatives).  The paper has no adjoint; this
 * is the differentiation form built on its step.  It runs in two calls, so
 * that a caller (an autograd function) can take the objective now and the
 * gradient later; kwgb_adjoint makes both calls.
 *
 * kwgb_adjoint_forward: run n_steps forward and return the objective.
 *   obj_idx    n_obj unique linear indices (host) of the objective region
 *   objective  KWGB_OBJ_MEAN_ABS_P (d|p|/dp taken as sign(p))
 *   n_steps    steps of the run (the simulation must not have stepped yet)
 *   checkpoint_every  0 < K < n_steps: keep the state every K steps
 *              (device memory ~ (n_steps/K) * 7 fields) for
 *              kwgb_adjoint_backward, which recomputes the steps between;
 *              K >= n_steps: keep every step's density fields instead
 *              (rho_xi, the Eq. 4c derivatives d_xi and the total density:
 *              7 fields, 28 N bytes a step), written by the forward steps
 *              themselves, so that the backward pass recomputes nothing
 *              (OOM if they do not fit: take a smaller K);
 *              K = 0: the objective only (no checkpoints, no gradient later)
 *   J_out      objective value (host)
 * The simulation then holds the end state (n_steps taken) and its sensors
 * the run's outputs.  Synchronises.  Errors: ARG, STATE (already stepped or
 * already run), UNSUPPORTED (K > 0 with a force or Dirichlet source: only
 * additive mass sources are differentiated), OOM, CUDA, NONFINITE. */
int kwgb_adjoint_forward(kwgb_sim* sim, const int64_t* obj_idx, int64_t n_obj, int objective,
                         int64_t n_steps, int64_t checkpoint_every, double* J_out, void* cuda_stream);

/* kwgb_adjoint_backward: the reverse pass of the run kwgb_adjoint_forward
 * made (checkpoint_every > 0).  With checkpoints, each K-step segment is
 * recomputed from its checkpoint, keeping rho_xi, the Eq. 4c derivatives
 * d_xi and the total density of every step (device memory ~ 7 K fields),
 * then stepped backwards; with every step kept, the steps are stepped
 * backwards directly.
 *   grad_out   host, grad_len doubles: for every source in add order, its
 *              n_signals rows of n_t values dJ/dsignal[row][n]
 * Afterwards the simulation holds the forward end state and sensor outputs
 * again.  Synchronises.  Errors: ARG (buffer too small), STATE (no pending
 * forward run), OOM, CUDA, NONFINITE. */
int kwgb_adjoint_backward(kwgb_sim* sim, double* grad_out, int64_t grad_len, void* cuda_stream);

/* Both calls in one: kwgb_adjoint_forward (checkpoint_every > 0) then
 * kwgb_adjoint_backward.  Errors as theirs. */
int kwgb_adjoint(kwgb_sim* sim, const int64_t* obj_idx, int64_t n_obj, int objective,
                 int64_t n_steps, int64_t checkpoint_every, double* J_out, double* grad_out,
                 int64_t grad_len, void* cuda_stream);

/* ---- checkpoint / restart of a run -------------------------------------
 * A snapshot holds everything a step reads and writes: u_xi, rho_xi, the
 * x-transformed pressure spectrum, every sensor accumulator (p_max, sum of
 * p^2, last p at masked points, full-grid maps, intensity sums) and the step
 * index.  Continuing from a snapshot is bitwise identical to not having
 * stopped.  The paper's code splits long runs into phases by saving the
 * time-varying fields and the aggregated outputs and reloading them
 * (Sec. 3.4, simulation stages); these calls are that facility for one GPU,
 * with the file I/O left to the caller.
 * The grid, medium, sources and sensors are not part of the snapshot: a
 * restore needs a simulation created and set up the same way (same
 * descriptor, medium, sources and sensors in the same order).  The first of
 * these calls freezes the source and sensor lists, as kwgb_step does. */

/* Bytes of a snapshot of sim (0 on error). */
int64_t kwgb_state_bytes(kwgb_sim* sim);

/* Copy the state into host memory buf (len >= kwgb_state_bytes bytes,
 * caller-owned).  Synchronises the device.  Errors: ARG (null or short
 * buffer), STATE (no medium), CUDA. */
int kwgb_save_state(kwgb_sim* sim, void* buf, int64_t len);

/* Restore a snapshot written by kwgb_save_state (buf is read only; len its
 * size).  The snapshot's grid and sensor layout must match sim's, else ARG;
 * the device status flag is cleared.  Synchronises.  Errors: ARG, STATE,
 * CUDA. */
int kwgb_load_state(kwgb_sim* sim, const void* buf, int64_t len);

/* Number of steps taken so far. */
int64_t kwgb_steps_done(const kwgb_sim* sim);

/* Kernels launched by the simulation so far (all calls). */
int64_t kwgb_launch_count(const kwgb_sim* sim);

/* One time step like kwgb_step(sim, 1, cuda_stream), with a CUDA event
 * recorded on cuda_stream after every kernel launch.  Synchronises.  Writes
 * for each launch, in order, its kernel kind (see kwgb_kernel_name) to
 * kinds[] and its device duration in milliseconds (from the previous event)
 * to ms[], at most capacity entries; *n_launches receives the count.  This is
 * the measurement hook of the benchmark.  Errors: ARG, STATE, CUDA. */
int kwgb_step_profiled(kwgb_sim* sim, void* cuda_stream, int32_t* kinds, float* ms,
                       int32_t capacity, int32_t* n_launches);

/* Name of a kernel kind reported by kwgb_step_profiled ("" if unknown).
 * The string is static. */
const char* kwgb_kernel_name(int32_t kind);

/* Synchronise and report device-side status: KWGB_OK, KWGB_ERR_NONFINITE
 * or KWGB_ERR_CUDA. */
int kwgb_status(kwgb_sim* sim);

/* Test hook of the failure path: with on != 0 every later tile load of the
 * y/z passes waits for 16 bytes more than it receives, so its bounded wait
 * (2 s) runs out; the kernels then skip their stores and return, and
 * kwgb_status reports KWGB_ERR_TIMEOUT (the CUDA context stays usable).
 * on = 0 restores normal loads.  No device fault, trap or hang is involved.
 * Errors: ARG. */
int kwgb_debug_wait_fault(kwgb_sim* sim, int on);

/* Device bytes held by the simulation. */
int64_t kwgb_device_bytes(const kwgb_sim* sim);

/* Message describing the last failure on sim ("" if none); with sim == NULL,
 * the last failure of kwgb_create.  Valid until the next call on sim. */
const char* kwgb_last_error(const kwgb_sim* sim);

/* Release the simulation and all its device memory.  NULL is a no-op. */
void kwgb_destroy(kwgb_sim* sim);

#ifdef __cplusplus
}
#endif

#endif /* KWGB_H */
