/*
 * fdbb.h -- C ABI of the GB300 (sm_103a) Euler building-block library.
 *
 * The library evaluates the compressible-Euler "building blocks" of FDBB
 * (M. Moeller, A. Jaeschke, "FDBB: Fluid Dynamics Building Blocks") point by
 * point over structure-of-arrays fields resident in GPU memory.  Every entry
 * point launches one fused CUDA kernel: it reads each input plane once, keeps
 * all intermediate values in registers and writes each output plane once.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - dim D in {1,2,3}; nv = D + 2 components per point.
 *  - Planes.  A field is an array of nv "planes"; plane k holds component k
 *    of all n points contiguously.  Callers pass a HOST array of DEVICE plane
 *    pointers.  Component order (paper, section 2.2, Figs. 7 and 9):
 *      conservative U = (rho, m_1..m_D, rhoE),  m = rho v,
 *      primitive    V = (rho, v_1..v_D, p).
 *    Flux Jacobians are nv*nv planes in row-major block order A[r*nv + c]
 *    (the default block storage order, paper section 2.1, "Block
 *    Expressions").
 *  - Storage type t applies to every plane of a call.  FDBB_F64 computes in
 *    IEEE double.  FDBB_F32 / FDBB_F16 / FDBB_BF16 compute in float and
 *    recover the internal energy rhoE - |m|^2/(2 rho) with compensated
 *    (error-free-transform) float arithmetic, so p stays accurate near vacuum
 *    and at high Mach; outputs are rounded to nearest-even into t.
 *  - gamma is the ratio of specific heats c_p / c_v (1.4 in the paper,
 *    section 2.2); derived constants (gamma - 1, 3 - gamma, 2/(gamma - 1))
 *    are formed on the host in double and then rounded once to the compute
 *    type.
 *  - Every plane pointer must be 16-byte aligned (the kernels use 128-bit
 *    loads and stores); n may be any value >= 0 (a ragged tail is handled).
 *  - Ownership: the caller owns all memory.  Entry points never allocate,
 *    free or synchronise; the kernel is enqueued on `stream` (NULL = the
 *    legacy default stream) and the call returns immediately.
 *  - Aliasing: an output plane may be the same pointer as an input plane of
 *    the same point index (in-place update, e.g. V written over U); any other
 *    overlap is undefined.
 *  - A NULL output plane pointer means "do not compute / write this output".
 *    Input plane pointers must not be NULL.
 *  - Errors: arguments are checked before anything is enqueued; on an
 *    argument error nothing is written and the corresponding status is
 *    returned.  A failed launch returns FDBB_ERR_CUDA (the CUDA error is
 *    consumed with cudaGetLastError).  n == 0 returns FDBB_OK without a
 *    launch.
 *  - Non-physical states (rho <= 0 or p < 0) are not clamped: the square
 *    root of a negative number gives NaN, which propagates.
 */
#ifndef FDBB_H
#define FDBB_H

#include <stdint.h>

#if defined(__GNUC__)
#define FDBB_API __attribute__((visibility("default")))
#else
#define FDBB_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t (the CUDA runtime's stream handle). */
typedef struct CUstream_st *fdbb_stream_t;

typedef enum {
  FDBB_OK = 0,
  FDBB_ERR_ARG = 1,     /* dim not in {1,2,3}, dir out of range, n < 0, gamma <= 1 */
  FDBB_ERR_NULLPTR = 2, /* a required plane array or input plane is NULL         */
  FDBB_ERR_ALIGN = 3,   /* a plane pointer is not 16-byte aligned                */
  FDBB_ERR_DTYPE = 4,   /* unknown storage type                                  */
  FDBB_ERR_CUDA = 5,    /* the kernel launch failed                              */
  FDBB_ERR_TIMEOUT = 6, /* a bounded host wait on the device ran out             */
  FDBB_ERR_NOMEM = 7    /* a caller-supplied buffer or budget is too small       */
} fdbb_status;

/*
 * Storage type of every plane of a call (and the arithmetic used):
 *   FDBB_F64    double planes, IEEE double arithmetic.
 *   FDBB_F32    float planes, float arithmetic (compensated rho e).
 *   FDBB_F16    half planes, float arithmetic (compensated rho e).
 *   FDBB_BF16   bfloat16 planes, float arithmetic (compensated rho e).
 *   FDBB_F64_DW double planes, double-word ("float-float", ~47-bit
 *               significand) arithmetic on the float pipe.  Results are within
 *               1e-12 of the running-error scale of each formula (the same
 *               bound the FDBB_F64 results meet).  A point where an input or a
 *               derived quantity (v, |v|^2/2, p, H, c^2) is non-zero with
 *               magnitude outside [2^-24, 2^24], or not finite, is computed in
 *               IEEE double instead.  Outputs that are copies of an input are
 *               bit-exact.  The inverse characteristic transforms form their
 *               sums of input weights (w_1 + w_2 + w_nv, w_nv - w_1, w_1 + w_nv)
 *               in IEEE double, the rest in double-word.  On GPUs whose FP64
 *               rate is a small fraction of the FP32 rate (GB300: 1/64) this is
 *               the fast FP64-storage form.
 */
typedef enum { FDBB_F64 = 0, FDBB_F32 = 1, FDBB_F16 = 2, FDBB_BF16 = 3, FDBB_F64_DW = 4 } fdbb_dtype;

/* Human-readable name of a status code (static string, never NULL). */
FDBB_API const char *fdbb_status_string(fdbb_status status);

/* Library version as an integer (major * 10000 + minor * 100 + patch). */
FDBB_API int fdbb_version(void);

/*
 * Kernels that stage their inputs through shared memory wait on the copies
 * with a bounded number of polls; a wait that runs out makes the kernel stop
 * (after waiting, bounded again, for its copies in flight) and count the
 * event.  fdbb_device_status synchronises with the device, returns
 * FDBB_ERR_TIMEOUT if any such wait ran out since the previous call (and
 * clears the count), else FDBB_OK.
 */
FDBB_API fdbb_status fdbb_device_status(void);

/*
 * Poll limit of the bounded waits above, for testing the failure path.
 * polls < 0 restores the default (2^22 polls per wait); polls >= 0 makes every
 * staged kernel launched afterwards, by any host thread, give up after that
 * many polls of each wait for its input copies (0: at the first wait, before
 * it computes or writes anything).  A kernel that gives up still waits, with
 * the default limit, for the copies it has issued, then returns; the next
 * fdbb_device_status reports FDBB_ERR_TIMEOUT.  Not meant for production use:
 * outputs of a launch that gave up are left unwritten.  Returns the previous
 * setting.
 */
FDBB_API int fdbb_set_wait_limit(int polls);

/*
 * Which kernel the calling host thread's most recent point-wise block launch
 * took (a diagnostic: the library picks the kernel from n, the storage type
 * and the device).
 *   kernel      FDBB_KERNEL_NONE (no launch yet on this thread),
 *               FDBB_KERNEL_DIRECT (plane loads straight from global memory),
 *               FDBB_KERNEL_STAGED (bulk asynchronous copies of 256-thread
 *               tiles into a two-stage shared-memory ring; ragged tail direct);
 *   grid, block blocks and threads per block of that launch;
 *   smem_bytes  its dynamic shared memory;
 *   points_per_thread  consecutive points each thread takes per plane (the
 *               tile of the staged kernel is block * points_per_thread points).
 * Host-side only; enqueues nothing.  FDBB_ERR_NULLPTR if info is NULL.
 */
typedef enum { FDBB_KERNEL_NONE = 0, FDBB_KERNEL_DIRECT = 1, FDBB_KERNEL_STAGED = 2 } fdbb_kernel_kind;
typedef struct fdbb_launch_info {
  int32_t kernel;
  int32_t grid;
  int32_t block;
  int32_t smem_bytes;
  int32_t points_per_thread;
  int32_t reserved;
} fdbb_launch_info;
FDBB_API fdbb_status fdbb_last_launch(fdbb_launch_info *info);

/*
 * Index checks of a debug build.  A library compiled with -DFDBB_DEBUG
 * (libfdbb_debug.so: python -m paper_1809_09851_gb300.build --debug) checks,
 * inside its kernels, every global-memory index of the point-wise blocks and
 * the finite-volume steps against the field's size, and every plane index
 * of the staged kernels' shared-memory ring against the planes staged,
 * before the access.  A violation is counted, the first offending index
 * kept, and the access skipped (a load reads a harmless value; nothing
 * traps).  fdbb_debug_index_faults synchronises with the device, returns the
 * number of violations since the previous call (and clears it), and stores
 * the first offending index in *first_index (-1 if none; first_index may be
 * NULL).  A release build compiles the checks out and returns -1; -2 means
 * the counters could not be read.
 */
FDBB_API int64_t fdbb_debug_index_faults(int64_t *first_index);

/*
 * Where a plane pointer lives, for callers that hand the blocks host memory:
 *   FDBB_PTR_DEVICE  memory of the current CUDA device (cudaMalloc, stream-ordered
 *                    pools; another device's memory is FDBB_PTR_OTHER);
 *   FDBB_PTR_HOST    page-locked host memory (cudaHostAlloc, cudaMallocHost,
 *                    cudaHostRegister) that the device reads and writes at the
 *                    same address (unified addressing): the kernels accept it
 *                    as plane memory and move it over the CPU-GPU link;
 *   FDBB_PTR_MANAGED managed memory (cudaMallocManaged);
 *   FDBB_PTR_OTHER   anything else (pageable host memory, invalid pointers).
 * Synchronous with respect to the host, enqueues nothing; the CUDA error of a
 * failed query is consumed.
 */
typedef enum { FDBB_PTR_OTHER = 0, FDBB_PTR_DEVICE = 1, FDBB_PTR_HOST = 2, FDBB_PTR_MANAGED = 3 } fdbb_ptr_kind;
FDBB_API fdbb_ptr_kind fdbb_pointer_kind(const void *p);

/*
 * |v|^2 = (m_1^2 + .. + m_D^2) / rho^2, the kinetic-energy sub-expression
 * used as micro-benchmark in the paper (section 3, Eq. (2)).
 * U: the first D+1 planes of a conservative field (rho, m_1..m_D); y: 1 plane.
 */
FDBB_API fdbb_status fdbb_v_mag2(int dim, int64_t n, fdbb_dtype t, const void *const *U, void *y,
                        fdbb_stream_t stream);

/*
 * Conservative -> primitive, V = (rho, v, p) with v = m / rho and
 * p = (gamma - 1)(rhoE - |m|^2 / (2 rho)) (paper section 2.2, Fig. 9,
 * V = varU::primitive(U)).  U: nv planes in; V: nv planes out.  If V[0] is
 * NULL or equals U[0] the density plane is not written (no bandwidth is
 * spent copying rho onto itself, as the paper notes for Fig. 9).
 */
FDBB_API fdbb_status fdbb_prim_from_cons(int dim, double gamma, int64_t n, fdbb_dtype t,
                                const void *const *U, void *const *V, fdbb_stream_t stream);

/*
 * Primitive -> conservative, m = rho v, rhoE = p / (gamma - 1) + rho |v|^2 / 2
 * (paper section 2.2, Fig. 9, U = varV::conservative(V)).  V: nv planes in;
 * U: nv planes out (U[0] skipped when NULL or equal to V[0]).
 */
FDBB_API fdbb_status fdbb_cons_from_prim(int dim, double gamma, int64_t n, fdbb_dtype t,
                                const void *const *V, void *const *U, fdbb_stream_t stream);

/*
 * Ideal-gas equation of state from conservative variables (paper section 2.2,
 * Fig. 7, varU::p(U); "Equations of state"): pressure p = (gamma - 1) rho e
 * and speed of sound c = sqrt(gamma p / rho).  U: nv planes; p, c: one plane
 * each, either may be NULL.
 */
FDBB_API fdbb_status fdbb_eos(int dim, double gamma, int64_t n, fdbb_dtype t, const void *const *U,
                     void *p, void *c, fdbb_stream_t stream);

/*
 * Riemann invariants along direction dir in [0, dim) (named in the paper,
 * section 1 and Fig. 1): w- = u - 2c/(gamma - 1), w+ = u + 2c/(gamma - 1) with
 * u = v_dir, and the entropy s = p / rho^gamma.  Each output may be NULL.
 */
FDBB_API fdbb_status fdbb_riemann_inv(int dim, int dir, double gamma, int64_t n, fdbb_dtype t,
                             const void *const *U, void *wm, void *wp, void *s,
                             fdbb_stream_t stream);

/*
 * Inviscid flux (paper section 2.2, "Inviscid Fluxes": the N_U x N_D tensor
 * F(U) = [rho v; rho v (x) v + I p; v (rhoE + p)]).  dir in [0, dim) writes
 * the column F_dir (nv planes); dir == -1 writes all columns, direction-major:
 * plane d*nv + k is component k of F_d (dim*nv planes).
 */
FDBB_API fdbb_status fdbb_flux(int dim, int dir, double gamma, int64_t n, fdbb_dtype t,
                      const void *const *U, void *const *F, fdbb_stream_t stream);

/*
 * Flux Jacobian A_dir = dF_dir / dU (named in the paper, section 1 and
 * section 2.2, "Inviscid Fluxes", as forthcoming), nv*nv planes, row-major,
 * rows and columns in U order.  Entries that are identically 0 or 1 are
 * still written when their plane pointer is not NULL.
 */
FDBB_API fdbb_status fdbb_flux_jac(int dim, int dir, double gamma, int64_t n, fdbb_dtype t,
                          const void *const *U, void *const *A, fdbb_stream_t stream);

/*
 * Characteristic transform at the local state (characteristic variables are
 * named in the paper, section 1 and Fig. 1).  inverse == 0: Y = L_dir(U) W;
 * inverse != 0: Y = R_dir(U) W, where the columns of R are the right
 * eigenvectors of A_dir ordered by eigenvalue u - c, u (entropy), u (shear,
 * tangential directions ascending), u + c:
 *   r_1 = (1, v - c e_dir, H - u c), r_2 = (1, v, |v|^2/2),
 *   r_{2+k} = (0, e_t, v_t), r_nv = (1, v + c e_dir, H + u c),
 * H = (rhoE + p)/rho, and L = R^{-1}.  U, W: nv planes in; Y: nv planes out.
 */
FDBB_API fdbb_status fdbb_char_transform(int dim, int dir, double gamma, int64_t n, fdbb_dtype t,
                                int inverse, const void *const *U, const void *const *W,
                                void *const *Y, fdbb_stream_t stream);

/*
 * One pass computing all fluxes, one Jacobian and one characteristic
 * transform (the paper's mini-app evaluates the 3D inviscid fluxes over
 * initialised U repeatedly, section 3): F = all dim flux columns
 * (dim*nv planes, direction-major as fdbb_flux with dir == -1),
 * A = A_dir_jac (nv*nv planes), Y = L_dir_jac(U) W (nv planes).  U and W are
 * read once.  F, A, Y (the arrays) or any plane in them may be NULL; W may be
 * NULL only if Y is NULL.
 */
FDBB_API fdbb_status fdbb_euler_fused(int dim, int dir_jac, double gamma, int64_t n, fdbb_dtype t,
                             const void *const *U, const void *const *W, void *const *F,
                             void *const *A, void *const *Y, fdbb_stream_t stream);

/*
 * fdbb_euler_fused over planes that may live in page-locked host memory
 * (FDBB_PTR_HOST, see fdbb_pointer_kind) as well as in device memory: the
 * kernel reads and writes host planes directly over the CPU-GPU link
 * (NVLink-C2C on Grace-Blackwell), so a field resident in host memory needs
 * no staging copies and no device memory.  Every non-NULL plane is checked
 * with fdbb_pointer_kind before the launch: a plane that is neither device
 * memory nor page-locked host memory returns FDBB_ERR_ARG and nothing is
 * enqueued.  When an input plane is host (or managed) memory the direct
 * kernel (plain global loads) runs, since the bulk-copy staging reads device
 * memory only.  Arguments, layout and results are those of fdbb_euler_fused.
 */
FDBB_API fdbb_status fdbb_euler_fused_host(int dim, int dir_jac, double gamma, int64_t n, fdbb_dtype t,
                                           const void *const *U, const void *const *W, void *const *F,
                                           void *const *A, void *const *Y, fdbb_stream_t stream);

/*
 * Vector-Jacobian product of the direction-dir flux: gU = A_dir(U)^T G
 * (the reverse-mode derivative of F_dir, for automatic differentiation).
 * U, G: nv planes in; gU: nv planes out.
 */
FDBB_API fdbb_status fdbb_flux_vjp(int dim, int dir, double gamma, int64_t n, fdbb_dtype t,
                          const void *const *U, const void *const *G, void *const *gU,
                          fdbb_stream_t stream);

/*
 * Primitive-variable forms (paper section 2.2, Fig. 9: the building blocks
 * evaluated from V = (rho, v, p) instead of U).
 * fdbb_flux_prim: the inviscid flux of fdbb_flux computed from V,
 *   F_d = (rho u, rho u v + p e_d, u (gamma/(gamma-1) p + rho |v|^2/2)),
 *   u = v_dir; dir == -1 writes all columns, direction-major.
 * fdbb_flux_jac_prim: B_dir = dF_dir/dV, nv*nv planes row-major, rows in U
 *   order, columns in V order:
 *   row 0: (u, rho at col 1+dir, 0);
 *   row 1+i: (u v_i, rho (delta_{j,dir} v_i + delta_{ij} u) at col 1+j, delta_{i,dir});
 *   row nv-1: (u |v|^2/2, delta_{j,dir} (gamma/(gamma-1) p + rho |v|^2/2)
 *              + rho u v_j at col 1+j, gamma/(gamma-1) u).
 * V: nv planes in; F / B: nv (dim*nv) / nv*nv planes out.
 */
FDBB_API fdbb_status fdbb_flux_prim(int dim, int dir, double gamma, int64_t n, fdbb_dtype t,
                                    const void *const *V, void *const *F, fdbb_stream_t stream);
FDBB_API fdbb_status fdbb_flux_jac_prim(int dim, int dir, double gamma, int64_t n, fdbb_dtype t,
                                        const void *const *V, void *const *B, fdbb_stream_t stream);

/*
 * Temperature of the perfect gas (paper section 2.2, "Equations of state":
 * the T_rhoe member of the EOS prototype, Fig. 10): T = e / c_v with the
 * specific internal energy e = (rhoE - |m|^2/(2 rho)) / rho.  cv > 0 is the
 * specific heat at constant volume (the paper's EOSidealGas<Cp = 7/2,
 * Cv = 5/2> gives gamma = 7/5 and R = Cp - Cv = 1, so T = p / rho).
 * U: nv planes in; T: one plane out.
 */
FDBB_API fdbb_status fdbb_temperature(int dim, double gamma, double cv, int64_t n, fdbb_dtype t,
                                      const void *const *U, void *T, fdbb_stream_t stream);

/*
 * Roe flux between two states per point (the step that follows the
 * point-wise blocks in a finite-volume solver; the paper names the inviscid
 * flux, section 2.2, and the characteristic variables, section 1):
 *   Fh = (F_dir(U_L) + F_dir(U_R))/2 - 1/2 R^ (|lambda^| * (L^ (U_R - U_L))),
 * where R^, L^ = R^{-1} and lambda^ are the eigenvectors and eigenvalues
 * defined at fdbb_char_transform, evaluated at the Roe-averaged state
 * (P. L. Roe, J. Comput. Phys. 43, 1981): with w = sqrt(rho),
 *   v^ = (w_L v_L + w_R v_R)/(w_L + w_R),  H^ likewise,
 *   c^2 = (gamma - 1)(H^ - |v^|^2/2).
 * No entropy fix.  U_L, U_R: nv planes each; F: nv planes.
 */
FDBB_API fdbb_status fdbb_roe_flux(int dim, int dir, double gamma, int64_t n, fdbb_dtype t,
                                   const void *const *UL, const void *const *UR, void *const *F,
                                   fdbb_stream_t stream);

/*
 * Characteristic transform at the Roe-averaged state of (U_L, U_R):
 * inverse == 0: Y = L^ W; inverse != 0: Y = R^ W.  U_L, U_R, W: nv planes
 * each; Y: nv planes.  (For FDBB_F64_DW the inverse runs in IEEE double.)
 */
FDBB_API fdbb_status fdbb_roe_char_transform(int dim, int dir, double gamma, int64_t n,
                                             fdbb_dtype t, int inverse, const void *const *UL,
                                             const void *const *UR, const void *const *W,
                                             void *const *Y, fdbb_stream_t stream);

/* ------------------------------------------------------------------------
 * General equations of state.
 *
 * The paper lets a user plug in an equation of state f(p, V, T) = 0 through a
 * type with members p_rhoe(rho, e) and T_rhoe(rho, e) (section 2.2,
 * "Equations of state", Fig. 10).  The entry points below evaluate the
 * EOS-dependent blocks under such a model instead of the ideal gas:
 *
 *   FDBB_EOS_NASG  Noble-Abel stiffened gas (Le Metayer and Saurel 2016),
 *                  p = (gamma - 1)(e - q) rho / (1 - b rho) - gamma p_inf,
 *                  T = (e - q - p_inf (1/rho - b)) / c_v
 *                  (the ideal gas for p_inf = b = q = 0; the stiffened gas for b = 0);
 *   FDBB_EOS_VDW   van der Waals with caloric law e = c_v T - a rho,
 *                  p = (gamma - 1)(rho e + a rho^2)/(1 - b rho) - a rho^2,
 *                  T = (e + a rho) / c_v;
 *   FDBB_EOS_IDEAL the ideal gas: the call runs the corresponding ideal-gas
 *                  entry point above with gamma and cv (every storage type).
 *
 * With the pressure gradient dp/dU = (phi, -Gamma v, Gamma), Gamma =
 * (1/rho) dp/de|_rho, phi = dp/drho|_e + Gamma (q - e), q = |v|^2/2, the
 * blocks are the ideal-gas ones with these per-point values in place of
 * gamma - 1 and (gamma - 1) q:
 *   c^2 = dp/drho|_e + Gamma p / rho (isentropic derivative),
 *   A_d: row 1+d = (phi - u^2, -Gamma v_j, (2 - Gamma) u, Gamma),
 *        row nv-1 = (u (phi - H), -Gamma u v_j, H - Gamma u^2, (1 + Gamma) u),
 *   eigenvectors as at fdbb_char_transform except the entropy wave
 *        r_2 = (1, v, 2q - phi/Gamma), L = R^{-1},
 *   rhoE = rho e(rho, p) + rho q in the primitive forms (whose Jacobian row
 *        nv-1 is (u (q + d(rho e)/drho|_p), delta_jd (rhoE + p) + rho u v_j,
 *        u (d(rho e)/dp|_rho + 1))).
 * The kernels take the partial derivatives of p(rho, e) and rho e(rho, p)
 * from one evaluation on dual numbers.
 *
 * Storage types: every one, as for the ideal gas: FDBB_F64 (IEEE double),
 * FDBB_F64_DW (double-word, with the same range rule and IEEE fallback; if an
 * EOS parameter (gamma - 1, its reciprocal, b, 1/c_v, p_inf, q, gamma p_inf,
 * a) is non-zero and outside [2^-24, 2^24] the call runs in IEEE double), and
 * FDBB_F32 / FDBB_F16 / FDBB_BF16 (float arithmetic with the compensated
 * internal energy, then the model's formulas in float).  The Riemann invariants and the
 * Roe-averaged forms have no counterpart here (no closed form for a general
 * EOS).  Argument errors (FDBB_ERR_ARG): eos NULL, unknown kind, gamma <= 1,
 * cv <= 0, b < 0, p_inf < 0 (NASG) or a < 0 (VDW).  States with
 * 1 - b rho <= 0 or c^2 < 0 are not checked: they give inf or NaN.
 * Every other convention (planes, alignment, NULL outputs, streams,
 * ownership) is that of the ideal-gas entry point of the same block.
 * ------------------------------------------------------------------------ */

typedef enum { FDBB_EOS_IDEAL = 0, FDBB_EOS_NASG = 1, FDBB_EOS_VDW = 2 } fdbb_eos_kind;

typedef struct fdbb_eos_model {
  int32_t kind;    /* fdbb_eos_kind */
  int32_t reserved; /* must be 0 */
  double gamma;    /* ratio of specific heats, > 1 */
  double p_inf;    /* NASG stiffening pressure, >= 0 */
  double b;        /* co-volume (NASG, VDW), >= 0 */
  double q;        /* NASG reference energy */
  double a;        /* VDW attraction, >= 0 */
  double cv;       /* specific heat at constant volume (temperature), > 0 */
} fdbb_eos_model;

/* Blocks under a general EOS: arguments as the ideal-gas entry point of the
 * same name without the suffix (gamma and cv come from the model). */
FDBB_API fdbb_status fdbb_prim_from_cons_eos(const fdbb_eos_model *eos, int dim, int64_t n, fdbb_dtype t,
                                             const void *const *U, void *const *V, fdbb_stream_t stream);
FDBB_API fdbb_status fdbb_cons_from_prim_eos(const fdbb_eos_model *eos, int dim, int64_t n, fdbb_dtype t,
                                             const void *const *V, void *const *U, fdbb_stream_t stream);
/* p and c (the block fdbb_eos computes for the ideal gas). */
FDBB_API fdbb_status fdbb_pressure_eos(const fdbb_eos_model *eos, int dim, int64_t n, fdbb_dtype t,
                                       const void *const *U, void *p, void *c, fdbb_stream_t stream);
/* T = T_rhoe(rho, e) of the model. */
FDBB_API fdbb_status fdbb_temperature_eos(const fdbb_eos_model *eos, int dim, int64_t n, fdbb_dtype t,
                                          const void *const *U, void *T, fdbb_stream_t stream);
FDBB_API fdbb_status fdbb_flux_eos(const fdbb_eos_model *eos, int dim, int dir, int64_t n, fdbb_dtype t,
                                   const void *const *U, void *const *F, fdbb_stream_t stream);
FDBB_API fdbb_status fdbb_flux_jac_eos(const fdbb_eos_model *eos, int dim, int dir, int64_t n, fdbb_dtype t,
                                       const void *const *U, void *const *A, fdbb_stream_t stream);
FDBB_API fdbb_status fdbb_char_transform_eos(const fdbb_eos_model *eos, int dim, int dir, int64_t n,
                                             fdbb_dtype t, int inverse, const void *const *U,
                                             const void *const *W, void *const *Y, fdbb_stream_t stream);
FDBB_API fdbb_status fdbb_euler_fused_eos(const fdbb_eos_model *eos, int dim, int dir_jac, int64_t n,
                                          fdbb_dtype t, const void *const *U, const void *const *W,
                                          void *const *F, void *const *A, void *const *Y, fdbb_stream_t stream);
FDBB_API fdbb_status fdbb_flux_vjp_eos(const fdbb_eos_model *eos, int dim, int dir, int64_t n, fdbb_dtype t,
                                       const void *const *U, const void *const *G, void *const *gU,
                                       fdbb_stream_t stream);
FDBB_API fdbb_status fdbb_flux_prim_eos(const fdbb_eos_model *eos, int dim, int dir, int64_t n, fdbb_dtype t,
                                        const void *const *V, void *const *F, fdbb_stream_t stream);
FDBB_API fdbb_status fdbb_flux_jac_prim_eos(const fdbb_eos_model *eos, int dim, int dir, int64_t n,
                                            fdbb_dtype t, const void *const *V, void *const *B,
                                            fdbb_stream_t stream);

/* ------------------------------------------------------------------------
 * Batched finite-volume steps (the serving workload).
 *
 * An explicit first-order finite-volume scheme with the Rusanov (local
 * Lax-Friedrichs) numerical flux built on the paper's inviscid flux
 * (section 2.2, "Inviscid Fluxes"), on periodic n^3 grids over [0,1]^3,
 * dx = 1/n, cell (i,j,k) at plane index (k*n + j)*n + i:
 *   Fh_d = (F_d(U_L) + F_d(U_R))/2 - s (U_R - U_L)/2,
 *          s = max(|v_d,L| + c_L, |v_d,R| + c_R);
 *   U_new = U - dt/dx * sum_d (Fh_{d,+1/2} - Fh_{d,-1/2});
 *   dt    = CFL * dx / max_cells sum_d (|v_d| + c), from the state at the
 *           start of the step.
 * The paper has no finite-volume scheme; this one is the standard
 * first-order scheme (Toro, ch. 10) driven by the paper's flux.
 *
 * Many grids of different sizes are advanced in one launch.  Each grid owns
 * a range of a virtual cell index space that starts at a multiple of
 * FDBB_FV_TILE and is FDBB_FV_TILE-padded; descriptors are passed in a HOST
 * array (copied into the launch), sorted by cell_begin, at most
 * FDBB_FV_MAX_GRIDS per call.  The per-grid maximum wave speed lives in a
 * caller-owned DEVICE scratch array `smax` of the storage type, three slots
 * per grid (smax[3*slot + 0..2]):
 *   fdbb_fv_max_speed   reduces max sum_d(|v_d| + c) of U into slot `phase`
 *                       (which the caller must have set to 0);
 *   fdbb_fv_rusanov_step reads slot `phase`, writes U_new, reduces U_new's
 *                       wave speed into slot (phase+1)%3 and clears slot
 *                       (phase+2)%3.
 * So a grid started with fdbb_fv_max_speed at phase 0 (slots zeroed) can be
 * stepped any number of times by incrementing phase modulo 3 and swapping U
 * and Unew between calls.  The maximum is order independent: a grid's
 * results do not depend on the other grids in the launch.
 * Storage: FDBB_F32 (float arithmetic with compensated internal energy) or
 * FDBB_F64 (double).  Arguments are checked on the host (ranges sorted,
 * aligned and inside vcells; planes non-NULL and aligned; Unew distinct from
 * U); device pointers themselves cannot be checked and must be valid.
 * Calls are asynchronous on `stream`; nothing is allocated.
 * ------------------------------------------------------------------------ */
#define FDBB_FV_TILE 256
#define FDBB_FV_MAX_GRIDS 256

typedef struct fdbb_fv_grid {
  void *U[5];         /* state at the start of the step (rho, m_x, m_y, m_z, rhoE), n^3 each */
  void *Unew[5];      /* state after the step (written by fdbb_fv_rusanov_step only)        */
  double *dt_log;     /* optional device array: dt of this step stored at dt_log[step]      */
  int64_t cell_begin; /* first virtual cell index, a multiple of FDBB_FV_TILE                */
  int32_t n;          /* cells per side, 1 <= n <= 4096                                     */
  int32_t slot;       /* wave-speed slots smax[3*slot .. 3*slot+2]                          */
  int32_t phase;      /* step index modulo 3                                                */
  int32_t step;       /* step index (position in dt_log)                                    */
} fdbb_fv_grid;

FDBB_API fdbb_status fdbb_fv_max_speed(int ngrids, const fdbb_fv_grid *grids, int64_t vcells,
                                       double gamma, fdbb_dtype t, void *smax, fdbb_stream_t stream);

FDBB_API fdbb_status fdbb_fv_rusanov_step(int ngrids, const fdbb_fv_grid *grids, int64_t vcells,
                                          double gamma, double cfl, fdbb_dtype t, void *smax,
                                          fdbb_stream_t stream);

/*
 * fdbb_fv_init_smooth -- smooth periodic initial state of one grid (the
 * requests of the serving workload; the paper has no counterpart):
 *   rho = 1 + amplitude * g_0 / max|g_0|,  v = 0,  p = 1 + amplitude * g_1 / max|g_1|,
 *   g_r(x) = sum_{m=0..2} a_{r,m} sin(2 pi (k_{r,m} . x) + phi_{r,m}),
 * at the cell centres x = ((i, j, k) + 1/2) / n, written as conservative
 * U = (rho, 0, 0, 0, p / (gamma - 1)) into grid->U (only U and n are read).
 * wave: HOST array of 30 doubles, (k_x, k_y, k_z, phi, a) of sinusoid m of
 * plane r at wave[15 r + 5 m].  scratch: DEVICE array of two values of the
 * storage type (the two maxima; overwritten).  Storage FDBB_F32 (evaluated in
 * float) or FDBB_F64.  One memset and two launches on `stream`.
 */
FDBB_API fdbb_status fdbb_fv_init_smooth(const fdbb_fv_grid *grid, double gamma, double amplitude,
                                         const double *wave, fdbb_dtype t, void *scratch,
                                         fdbb_stream_t stream);

/*
 * fdbb_fv_rusanov_step_noalloc -- the same step for callers that cannot
 * allocate device memory.  (The paper has no counterpart; this is an
 * interface convenience of this library.)
 *
 * Some callers cannot call cudaMalloc: host frameworks that own every byte of
 * device memory and hand plug-ins only the buffers they manage, or time-
 * critical loops where an allocation (which may synchronise the device) is not
 * allowed.  They still pass the grid state (U, Unew, dt_log) as with
 * fdbb_fv_rusanov_step, but no wave-speed scratch: this entry point keeps it
 * in a fixed array of the library's own device memory, 3 * FDBB_FV_MAX_GRIDS
 * doubles (6 KiB), which every GPU that loads the library holds until the
 * process exits.  Nothing is allocated or freed by the call.
 *
 * Each call is one complete step: it clears the array, reduces the maximum
 * wave speed of every grid's U into it and advances the grids, so the
 * descriptors' `slot` and `phase` fields are ignored (dt is still that of the
 * state at the start of the step, and dt_log[step] is written as usual).  The
 * results equal those of fdbb_fv_max_speed + fdbb_fv_rusanov_step.
 * At most FDBB_FV_MAX_GRIDS grids per call; more returns FDBB_ERR_ARG.
 * The grid table is checked first (as in fdbb_fv_rusanov_step); a call with
 * invalid arguments returns its error before any CUDA call.  The first valid
 * call on a device then looks up the array's device address
 * (cudaGetSymbolAddress, once per device, with that device current) and
 * caches it for the rest of the process; make that first call before any
 * stream capture.  The cached address belongs to the device's context at that
 * time: after cudaDeviceReset of that device the library's module is loaded
 * again and the address may change, so a process that resets a device must
 * not call this entry point on that device again.  All calls share the array
 * and it keeps the last call's contents, so calls that overlap on the GPU (on
 * different streams, or from different threads) race: serialise them.
 */
FDBB_API fdbb_status fdbb_fv_rusanov_step_noalloc(int ngrids, const fdbb_fv_grid *grids,
                                                  int64_t vcells, double gamma, double cfl,
                                                  fdbb_dtype t, fdbb_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* FDBB_H */
