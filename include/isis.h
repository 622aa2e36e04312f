/*
 * isis.h -- C ABI of the GB300 library for the scalar-field multigrid solve
 * of ISIS (Llinares, Mota & Winther 2013, "ISIS: a new N-body cosmological
 * code with scalar fields based on RAMSES", arXiv:1307.6748).
 *
 * The paper states the problem as (Sect. 1, Eqs. (eqs_general_1)-(eqs_general_3)):
 *     lap Phi  = (3/2) Omega_m H0^2 delta / a                 (Newtonian potential)
 *     lap phi  = S(phi, rho, a)                               (scalar field, quasi-static)
 *     x''      = -grad Phi / a^2 - g(phi, grad phi, a)        (particles)
 * and this library solves them on a periodic, cell-centred N^3 grid:
 *     isis_cic_deposit    particles -> density eta (Sect. 5.1, "CIC")
 *     isis_poisson_solve  lap Phi = (3/2) Om H0^2 (eta - <eta>) / a (Sect. 3.1)
 *     isis_scalar_solve   L(phi, eta) = 0 by non-linear FAS multigrid with
 *                         Newton-Gauss-Seidel smoothing (Sect. 3.2) for the
 *                         symmetron (Sect. 4.1) or Hu-Sawicki f(R) (Sect. 4.2)
 *     isis_fifth_force    gradients interpolated back to particles
 *                         (Sect. 4.1 Eq. (symmetron_geodesics_tilde_chi), Sect. 4.2)
 *
 * Conventions shared by every call
 *   - Grid: N^3 cells, N a power of two, 8 <= N <= 1024, cell (i,j,k) at
 *     index (i*N + j)*N + k (k fastest), centre at (i+1/2, j+1/2, k+1/2) h,
 *     h = box / N, periodic in all directions.
 *   - Units: lengths in Mpc/h, c = 1, so H0 = 1/2997.92458 per Mpc/h.
 *   - Memory: every array argument is a DEVICE pointer owned by the caller,
 *     contiguous, on the current CUDA device; the library never frees or
 *     keeps it.  The library owns its level hierarchy (workspace), cached
 *     per grid size and precision until isis_release_workspace().
 *   - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy
 *     default stream).  Work is stream ordered.  The solvers synchronise the
 *     stream once per cycle to read the residual norm; deposit and force
 *     calls do not synchronise.
 *   - Errors: every call returns an isis_status; nothing aborts.  Calls are
 *     not thread safe (one host thread drives the library at a time).
 */
#ifndef ISIS_H
#define ISIS_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ISIS_OK = 0,
  ISIS_EINVAL = -1,    /* bad argument: sizes, pointers, parameters */
  ISIS_ENOCONV = -2,   /* max_cycles reached, or a coarsest-grid Newton solve met no stop within its 50
                          steps (that cycle then ends the solve); last iterate left in phi, info filled */
  ISIS_ENAN = -3,      /* non-finite residual or a singular coarsest Jacobian */
  ISIS_ECUDA = -4,     /* a CUDA runtime call or launch failed */
  ISIS_ENOMEM = -5,    /* device allocation of the workspace failed */
  ISIS_ETIMEOUT = -6,  /* reserved: a bounded device wait gave up */
  ISIS_EINTERNAL = -7
} isis_status;

typedef enum { ISIS_SYMMETRON = 1, ISIS_FOFR_HS = 2, ISIS_CHAMELEON = 3 } isis_model;

/* Arithmetic of a solve.
 *   ISIS_F64           eta, phi are double; every kernel computes in FP64.
 *   ISIS_F32           eta, phi are float; every kernel computes in FP32
 *                      (coarsest dense Newton in FP64).
 *   ISIS_F32_REFINE64  eta, phi are double.  First FP32 FAS V-cycles on the
 *                      field itself until its residual is below 2e-4 of the
 *                      reference (or stops falling); then defect correction to
 *                      FP64 accuracy: the residual r = -L(phi) and the update
 *                      phi += e in float-float (two floats per value, about 48
 *                      significant bits, the field carried in that form), and e
 *                      solves L(phi + e) - L(phi) = r by FP32 FAS V-cycles on the
 *                      correction (inner_cycles per outer iteration; coarsest
 *                      dense Newton in FP64).  phi is written in FP64 on return. */
typedef enum { ISIS_F64 = 0, ISIS_F32 = 1, ISIS_F32_REFINE64 = 2 } isis_precision;

typedef struct {
  double Omega_m, Omega_L; /* density parameters */
  double H0;               /* Hubble constant in (Mpc/h)^-1, c = 1: 1/2997.92458 */
  double box;              /* box side in Mpc/h */
  int N;                   /* cells per dimension */
} isis_grid;

typedef struct {
  double lambda0, beta, a_ssb; /* symmetron (Sect. 4.1): range in Mpc/h, coupling, a at symmetry breaking */
  int n;                       /* Hu-Sawicki exponent (Sect. 4.2), n >= 1 */
  double fR0_abs;              /* |f_R0| */
  double cham_n;               /* chameleon exponent, -1 < n <= 8 (ISIS_CHAMELEON; lambda0 and beta as above) */
} isis_params;

/* Initial guess of a solve.
 *   ISIS_INIT_INPUT       phi holds the guess on entry.
 *   ISIS_INIT_BACKGROUND  phi is overwritten with the uniform background field:
 *                         chi_bg = sqrt(max(0, 1 - (a_SSB/a)^3)), u_bg = ln(a^2 |fbar_R(a)|)
 *                         with |fbar_R(a)| = |f_R0| [(1+4r)/(a^-3+4r)]^(n+1), r = OL/Om, Phi = 0.
 *   ISIS_INIT_LOCAL       phi is overwritten cell by cell with the solution for a
 *                         uniform density equal to the cell's eta (same formulas with
 *                         (a_SSB/a)^3 eta and eta a^-3); Phi = 0.  Suits f(R) with
 *                         dense haloes, where Newton steps from the background overshoot.
 *   ISIS_INIT_PARENT      refinement patches only: the unknowns start from the parent
 *                         field interpolated to them. */
typedef enum { ISIS_INIT_INPUT = 0, ISIS_INIT_BACKGROUND = 1, ISIS_INIT_LOCAL = 2, ISIS_INIT_PARENT = 3 } isis_init;

typedef struct {
  int nu1, nu2;        /* pre- and post-smoothing sweeps (red then black) per level */
  int n_coarsest;      /* coarsest grid size: 2 or 4 (dense Newton there) */
  int max_cycles;      /* cap on V-cycles (inner cycles for F32_REFINE64), <= 128 */
  isis_precision prec;
  int inner_cycles;    /* F32 V-cycles per FP64 outer iteration (F32_REFINE64), >= 1 */
  isis_init init;      /* initial guess */
  int fmg;             /* ISIS_F32_REFINE64: 1 starts the FP32 phase with nested iteration (full multigrid):
                          the guess restricted to every level, the coarsest level's own problem solved,
                          then on each finer level the coarse correction prolongated onto the restricted
                          guess and one V-cycle; counted as one cycle, and followed by a plain V-cycle
                          before the first residual norm.  0: plain V-cycles.  Not in the paper
                          (its solver starts each level's V-cycles from a guess, Sect. 3.2). */
} isis_mg_opts;

typedef struct {
  int cycles;          /* V-cycles run (all FP32 cycles for F32_REFINE64) */
  int outer;           /* FP64 outer iterations (F32_REFINE64), else 0 */
  int nhist;           /* entries of hist */
  double res0;         /* RMS residual of the initial guess (FP32-evaluated for F32_REFINE64) */
  double res_ref;      /* reference residual (below) */
  double res_final;    /* RMS residual on return (FP64-evaluated unless ISIS_F32) */
  double hist[128];    /* RMS residual after each V-cycle; for F32_REFINE64 after each FP32
                          field-form cycle, then after each FP64 outer iteration */
} isis_solve_info;

/* Convergence test of both solvers (the paper gives none): stop when
 *     RMS over the finest grid of L(phi) <= tol * res_ref,
 * res_ref = RMS of L(phi_bg) for the uniform background field phi_bg:
 *   symmetron  A s chi_bg * RMS(eta - 1), chi_bg = sqrt(max(0, 1 - (a_SSB/a)^3)),
 *              A = a^2/(2 lambda0^2), s = (a_SSB/a)^3
 *   f(R)       Om a H0^2 * RMS(eta - 1)
 *   Poisson    (3/2) Om H0^2 / a * RMS(eta - <eta>)
 * and res_ref = res0 when that is 0 (uniform density, or a < a_SSB). */

/* CIC density estimate (Sect. 5.1): eta[cell] = sum_p W(x_p - cell) / nbar,
 * nbar = npart / N^3, trilinear cloud-in-cell weights, periodic.
 *   x, y, z  device float[npart], positions in CELL units (a position is
 *            wrapped into [0, N)); cell centres at i + 1/2.
 *   eta      device double[N^3] (eta_f64 != 0) or float[N^3] (eta_f64 == 0),
 *            overwritten.
 * Accumulation is in 64-bit fixed point: each particle's eight weights are
 * truncated to multiples of 2^-40 and summed as unsigned integers, so the
 * result does not depend on the order of particles.  A cell's accumulator
 * holds less than 2^24 unit weights (2^64 / 2^40): the weights a cell
 * collects, (npart / N^3) times its overdensity eta, must stay below 2^24
 * (16.7 million particles), or that cell wraps silently; npart < 2^24 rules
 * it out for any clustering.  Uses an int64 N^3 scratch buffer cached by the
 * library.  EINVAL: npart < 1, npart > 2^40 or N invalid. */
isis_status isis_cic_deposit(const isis_grid* grid, const float* x, const float* y, const float* z, int64_t npart,
                             void* eta, int eta_f64, void* stream);

/* The same CIC deposit for callers that must not allocate device memory once
 * they are running: services held to a fixed device-memory budget, programs
 * whose device memory is owned by another allocator (a framework's caching
 * pool), and paths where the device-wide synchronisation that cudaMalloc and
 * cudaFree imply is not acceptable.  It has no counterpart in the paper.
 *   - Scratch: a fixed array of 64^3 int64 accumulators (2 MiB) compiled into
 *     the library; every GPU that loads the library holds it until the
 *     process exits.  Nothing is allocated or freed by this call.
 *   - Limits: grid->N <= 64 and npart < 2^24 (then no cell can collect the
 *     2^24 unit weights that would wrap its accumulator, however the particles
 *     cluster); larger grids or more particles return ISIS_EINVAL (use
 *     isis_cic_deposit).  Other arguments as for isis_cic_deposit, same result.
 *   - Device contexts: the array's address is cached per device for the life
 *     of the process; a device reset (cudaDeviceReset) invalidates it and is
 *     not supported between calls.
 *   - Set-up: the first call on each device looks up the array's device
 *     address (cudaGetSymbolAddress) with that device current; make that first
 *     call before any stream capture.
 *   - Sharing: all calls share the one array and each call clears the part it
 *     uses before accumulating, so calls must not overlap on the GPU (two calls
 *     on different streams without ordering between them race). */
isis_status isis_cic_deposit_noalloc(const isis_grid* grid, const float* x, const float* y, const float* z,
                                     int64_t npart, void* eta, int eta_f64, void* stream);

/* Newtonian potential (Sect. 3.1, Eq. (disc_lap), Eq. (explicit)):
 *     (sum of 6 neighbours - 6 Phi)/h^2 = (3/2) Om H0^2 (eta - <eta>) / a
 * solved by multigrid V-cycles with Gauss-Seidel smoothing (the Newton step
 * of Sect. 3.2 reduces to Eq. (explicit) for this linear operator); the
 * mean of Phi is set to 0 after every cycle.
 *   eta  device double[N^3] (float for ISIS_F32), mean density 1 expected.
 *   Phi  device double[N^3] (float for ISIS_F32): initial guess in, solution out.
 *   opts NULL for the defaults {2, 2, 4, 100, ISIS_F64, 2, ISIS_INIT_INPUT, 0}; info may be NULL. */
isis_status isis_poisson_solve(const isis_grid* grid, double a, const void* eta, void* Phi, double tol,
                               const isis_mg_opts* opts, isis_solve_info* info, void* stream);

/* Uniform background field of a scalar model at expansion factor a: the solution at eta = 1 everywhere, the
 * value ISIS_INIT_BACKGROUND writes as the initial guess.
 *   ISIS_SYMMETRON  chi_bg = sqrt(max(0, 1 - (a_SSB/a)^3))      (Sect. 4.1: the minimum of the effective
 *                   potential at the background density; 0 before symmetry breaking)
 *   ISIS_FOFR_HS    u_bar = ln(a^2 |fbar_R(a)|), |fbar_R(a)| = |f_R0| [(1 + 4r)/(a^-3 + 4r)]^(n+1),
 *                   r = Omega_L/Omega_m                         (Sect. 4.2, the f_R equation at eta = 1)
 *   ISIS_CHAMELEON  u = 3 ln(a) / (1 + n)                       (Sect. 6, the minimum at a^-3 eta = psi^-(1+n))
 *   out  host double, written on ISIS_OK.  Host arithmetic only: no device work, no stream.
 *   Returns ISIS_EINVAL for a NULL pointer, a <= 0 or parameters outside the solver's range. */
isis_status isis_background_field(isis_model model, const isis_params* params, const isis_grid* grid, double a,
                                  double* out);

/* Scalar field (Sect. 3.2, FAS with implicit Newton-Gauss-Seidel):
 *   ISIS_SYMMETRON  phi = chi:  lap chi = a^2/(2 lambda0^2) [ (a_SSB/a)^3 eta chi - chi + chi^3 ]
 *                   (Sect. 4.1, Eq. (symmetron_dimensionles))
 *   ISIS_FOFR_HS    phi = u, f_R = -a^-2 e^u:
 *                   div(e^u grad u) = Om a H0^2 (eta - 1)
 *                       - Om a^4 H0^2 (1 + 4 OL/Om)(|f_R0| a^2)^{1/(n+1)} e^{-u/(n+1)}
 *                       + Om a H0^2 (1 + 4 a^3 OL/Om)                  (Sect. 4.2)
 *                   discretised in flux form with face b = arithmetic mean
 *                   (Sect. 3.4, Eq. (disc_non_canonical)).
 *   ISIS_CHAMELEON  the chameleon equation of Sect. 6, lap phi = -M^{4+n} phi^{-(1+n)} + beta rho / M_pl,
 *                   as one more free source S (Sect. 2): with phi = phi_0 psi (phi_0 the minimum in
 *                   today's background) and phi = u = ln psi,
 *                   div(e^u grad u) = a^2 / ((1+n) lambda0^2) [a^-3 eta - e^{-(1+n) u}],
 *                   lambda0 = params->lambda0 the range of the field in today's background and
 *                   n = params->cham_n; the f(R) operator with other constants (n = -1/2 is the
 *                   Hu-Sawicki n = 1 model of Sect. 6's mapping).  Background u = 3 ln(a) / (1+n).
 *   eta  device array (double, or float for ISIS_F32) of eta = rho / mean rho.
 *   phi  device array of the same type: initial guess in, solution out (the
 *        symmetron's zero field is a fixed point: start from a positive guess).
 *   On ENOCONV the last iterate is in phi and info is filled. */
isis_status isis_scalar_solve(isis_model model, const isis_params* params, const isis_grid* grid, double a,
                              const void* eta, void* phi, double tol, const isis_mg_opts* opts,
                              isis_solve_info* info, void* stream);

/* Per-particle acceleration in super-comoving units (Sects. 4.1, 4.2):
 *     g = -[ grad Phi~ + F5 ],  Phi~ = a^2 Phi
 *     ISIS_SYMMETRON  F5 = 6 Om H0^2 (beta lambda0)^2 / a_SSB^3  chi~ grad chi~,  chi~ = a chi
 *     ISIS_FOFR_HS    F5 = (1/2) e^u grad u
 *     ISIS_CHAMELEON  F5 = a^2 grad(beta phi / M_pl) = a^2 3 (1+n) beta^2 Om H0^2 lambda0^2 e^u grad u
 * Gradients are 2-point central differences at cells, interpolated to the
 * particles with the CIC weights of isis_cic_deposit.
 *   Phi, phi    device arrays (double if fields_f64, else float); either may be
 *               NULL to leave its term out (model is ignored when phi is NULL).
 *   x, y, z     device float[npart], cell units.
 *   gx, gy, gz  device float[npart], overwritten.  */
isis_status isis_fifth_force(isis_model model, const isis_params* params, const isis_grid* grid, double a,
                             const void* Phi, const void* phi, int fields_f64, const float* x, const float* y,
                             const float* z, int64_t npart, float* gx, float* gy, float* gz, void* stream);

/* One leapfrog step of the particles in super-comoving time tau (Eqs. (leap_frog_1)
 * to (leap_frog_3)), fused kick and drift, positions and velocities in cell units:
 *     v += kick * g / h,   x += drift * v,   x wrapped into [0, N),   h = box / N.
 *   g       the acceleration of isis_fifth_force at the current positions (per Mpc/h).
 *   kick    (dtau_prev + dtau) / 2: the second half-kick of the previous step merged with
 *           the first of this one, as the paper reuses the second velocity evaluation
 *           (dtau_prev = 0 on the first step; a last half-kick dtau/2 synchronises).
 *   drift   dtau.  tau is measured in Mpc/h (c = 1): dtau = da / (a^3 H0 E(a)).
 *   x, y, z, vx, vy, vz  device float[npart], updated in place; gx, gy, gz read.
 *   EINVAL: bad grid, NULL pointers, npart < 1 or non-finite kick or drift. */
isis_status isis_kick_drift(const isis_grid* grid, float* x, float* y, float* z, float* vx, float* vy, float* vz,
                            const float* gx, const float* gy, const float* gz, int64_t npart, double kick,
                            double drift, void* stream);

/* ---- Refinement patches (Sect. 3.3.1, Sect. 3.4.1) ------------------------
 * One refinement level over a box of its parent grid, solved with the parent
 * field as boundary data, as the paper solves each refined level after its
 * parent.  The box is n[0] x n[1] x n[2] parent cells at `origin`, refined by
 * two: the patch arrays hold all (2n[0]) x (2n[1]) x (2n[2]) fine cells in
 * row-major order (k fastest), fine cell (i,j,k) centred at parent-cell
 * coordinates origin + (i+1/2, j+1/2, k+1/2)/2 and of size
 * h = grid->box / (grid->N 2^level).  `flags` marks the refined parent cells;
 * their children are the unknowns.  The other fine cells do not exist in the
 * paper's sense: they get the parent field by cell-centred trilinear
 * interpolation (weights 3/4, 1/4 per axis) and serve as boundary values.
 * Masks and ghost values follow the paper: mask +1 at unknowns and -1
 * elsewhere, restricted (mean of 8) on the patch's coarser multigrid levels,
 * and a masked neighbour of an unknown c enters the stencil as
 *     u_nb + (m_nb/m_c)(u_c - u_c^Pre)                         (Eq. (ueq))
 * with u_c^Pre the value of c when the smoothing phase began, b and db/du of
 * f(R) taken at that ghost value, and the Newton derivative gaining the terms
 * through it.  The converged field satisfies the equation at every unknown
 * with the boundary cells at their interpolated values.
 *   n          each even and >= 4; the coarsest level of the patch's multigrid
 *              (halving while all dimensions are even and the smallest >= 8)
 *              must have at most 32768 cells.
 *   origin     box origin in parent cells.
 *   parent_dims, parent_periodic
 *              level 1: the parent is the periodic domain grid (N, N, N), and the
 *              box may wrap round it; level >= 2: the parent is the previous
 *              patch's field (its fine dims) and 1 <= origin, origin + n + 1 <=
 *              parent_dims (the interpolation reads one parent cell beyond the box).
 *   eta_mean   Poisson: the domain's mean density (the source is K (eta - eta_mean)).
 *   flags      device uint8[n0 n1 n2]; flags on the outer layer of the box are rejected.
 *   parent     device double, parent_dims.
 *   eta, phi   device double[(2n0)(2n1)(2n2)]: the density of the patch cells, and
 *              the field: the guess at the unknowns in (ISIS_INIT_INPUT) or ignored
 *              (ISIS_INIT_PARENT); out, the solution at the unknowns and the
 *              interpolated parent elsewhere.
 *   opts       prec ISIS_F64, or ISIS_F32_REFINE64: the FP64 residual r = -L(u)
 *              at the unknowns, then inner_cycles FP32 V-cycles of the same patch
 *              FAS on the correction e about B = fp32(u), L(B + e) - L(B) = r,
 *              with masked neighbours entering as B_nb + e_nb + (m_nb/m_c)
 *              (e_c - e_c^Pre), then u += e; repeated until the FP64 residual
 *              meets the test (cycles counts the FP32 V-cycles, outer the FP64
 *              iterations, hist the FP64 residual after each; fmg is ignored).
 *              ISIS_F32 is rejected.  init ISIS_INIT_INPUT or ISIS_INIT_PARENT;
 *              n_coarsest is ignored.  The convergence test is the solvers' own
 *              over the unknowns (res_ref from the unknowns' eta).
 *   Workspace: allocated stream-ordered per call and freed before return.  The
 *   call synchronises the stream once to check the flags, then once per cycle
 *   (ISIS_F64) or per outer iteration (ISIS_F32_REFINE64). */
typedef struct {
  int n[3];
  int origin[3];
  int parent_dims[3];
  int parent_periodic;
  int level;
  double eta_mean;
} isis_patch;

isis_status isis_patch_poisson_solve(const isis_grid* grid, double a, const isis_patch* box, const void* parent,
                                     const uint8_t* flags, const void* eta, void* Phi, double tol,
                                     const isis_mg_opts* opts, isis_solve_info* info, void* stream);

isis_status isis_patch_scalar_solve(isis_model model, const isis_params* params, const isis_grid* grid, double a,
                                    const isis_patch* box, const void* parent, const uint8_t* flags,
                                    const void* eta, void* phi, double tol, const isis_mg_opts* opts,
                                    isis_solve_info* info, void* stream);

/* ---- Instrumentation (not part of the paper's method) -------------------
 * Every kernel launch of the library is counted.  When profiling is on, each
 * launch is also bracketed by CUDA events on its stream and its algorithmic
 * bytes (the minimum DRAM traffic of its work) are recorded, per kernel kind. */
typedef struct {
  const char* name;   /* kernel kind, e.g. "smooth_fine"; the multigrid kernels' kinds carry the model
                         and form of their instantiation, e.g. "smooth_fine[fofr/delta]" (a string owned
                         by the library, valid until it is unloaded) */
  int64_t launches;   /* launches recorded since the last reset */
  double ms;          /* summed event time of those launches */
  double bytes;       /* summed algorithmic bytes of those launches */
} isis_prof_entry;

/* on != 0: record events for every launch from now on. */
void isis_prof_enable(int on);
/* Zero the counters and drop recorded events. */
void isis_prof_reset(void);
/* Synchronise the device, then fill up to max entries (one per kernel kind,
 * and per model and form for the multigrid kernels, with at least one
 * launch); returns the number filled. */
int isis_prof_read(isis_prof_entry* out, int max);
/* Kernel launches issued by the library since the last isis_prof_reset(). */
int64_t isis_launch_count(void);

/* Human-readable name of a status code (static string). */
const char* isis_strerror(isis_status status);

/* Free every cached workspace buffer (synchronises the device first). */
void isis_release_workspace(void);

/* Page-locked HOST memory for the arrays that cross the host link every step (the particle positions given
 * to isis_cic_deposit and isis_fifth_force, the forces read back), so that their copies run as asynchronous
 * DMA on a stream.  bytes > 0; on success *out is a buffer of at least `bytes` bytes, zero-filled, owned by
 * the caller until isis_host_free(*out).  A buffer of at least one transparent huge page starts on a huge-page
 * boundary and is advised MADV_HUGEPAGE before its pages are touched (the copy engines' address translations
 * then cover it with a few entries); smaller buffers, or a kernel that grants no huge pages, get base pages.
 * Returns ISIS_EINVAL for out == NULL or bytes == 0, ISIS_ENOMEM when the mapping fails and ISIS_ECUDA when
 * the CUDA driver refuses to page-lock it (nothing is left allocated then).  Thread safe. */
isis_status isis_host_alloc(size_t bytes, void** out);
/* Unlock and unmap a buffer of isis_host_alloc; NULL is a no-op.  Returns ISIS_EINVAL for a pointer that
 * isis_host_alloc did not return (or that was freed already), ISIS_ECUDA when the driver's unregistration
 * fails (the buffer is unmapped all the same).  Thread safe. */
isis_status isis_host_free(void* ptr);

/* Self-test of the float-float exponential used by the f(R) residual of the
 * FP64 defect correction (table-driven, after Tang, ACM TOMS 1989): y[i] =
 * exp(x[i]) evaluated in float-float from x[i] rounded to float-float, for
 * |x| < 20.  x, y: device arrays of n doubles; stream ordered. */
isis_status isis_selftest_exp_ff(const double* x, double* y, int n, void* stream);

/* Self-test of the conversion that writes the carried float-float field back to FP64 at the end of a mixed
 * solve: out[i] = hl[2i] + hl[2i+1] rounded to nearest even, as one FP64 addition of the two floats would give
 * it, formed by integer operations; zero, subnormal, Inf and NaN high parts, and subnormal low parts, are
 * flushed as the library's FP32-to-FP64 conversion flushes them (zero, subnormal: a signed zero).  The pair
 * must be normalised (|lo| <= ulp(hi)/2) for the integer path; other pairs take an FP64 addition.  hl: device
 * array of 2n floats, out: device array of n doubles; stream ordered. */
isis_status isis_selftest_ff_to_f64(const float* hl, double* out, int n, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* ISIS_H */
