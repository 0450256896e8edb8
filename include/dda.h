/*
 * dda.h -- C ABI of the GB300 discrete-dipole-approximation (DDA) library.
 *
 * The library computes the hot path of the DDA as described in the DDSCAT 7.1
 * User Guide (Draine & Flatau 2010): for N polarizable points on a cubic
 * lattice it solves A P = E (guide, eq. AP=E, section "Choice of Iterative
 * Algorithm"), where the off-diagonal part of A is applied as a zero-padded
 * 3-D FFT convolution of the six independent components of the symmetric
 * dipole-dipole tensor with the three components of P (the method of Goodman,
 * Draine & Flatau 1991 that the guide's FFT options implement; guide, "Choice
 * of FFT Algorithm"), followed by a pointwise 3x3 complex multiply in Fourier
 * space.  Units: lattice spacing d = 1, Gaussian units, exp(-i omega t), |E0| = 1.
 *
 * Conventions shared by every entry point
 *  - All functions return a dda_status; DDA_OK is 0.  On any other status,
 *    dda_last_error() returns a message describing the failure.  No exception,
 *    abort or trap crosses this boundary.
 *  - Host arrays are read (or written) during the call only; the caller keeps
 *    ownership.  Device buffers ("_dev") are borrowed: the caller allocates
 *    them on the context's device and keeps them alive until the enqueued work
 *    has finished.  The context owns everything else (Green tensor, plans,
 *    workspaces) and frees it in dda_destroy.
 *  - Work is enqueued on the context's stream.  Calls that return host values
 *    (dda_solve, dda_cross_sections) synchronize that stream before returning.
 *  - Complex vectors over the target use the layout [rhs][3][N]: right-hand
 *    side (orientation-major, then polarization), Cartesian component of the
 *    Target Frame, then the occupied site in x-fastest lexicographic order of
 *    its lattice index (the order dda_get_sites returns).  Elements are
 *    interleaved (re, im) pairs of float (DDA_C64) or double (DDA_C128).
 *  - Calling an entry point before the state it needs exists returns
 *    DDA_ESTATE (order: target -> incident -> {green, polarizability} ->
 *    matvec / solve / cross sections).
 */
#ifndef DDA_GB300_H
#define DDA_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define DDA_API __attribute__((visibility("default")))
#else
#define DDA_API
#endif

typedef struct dda_ctx dda_ctx;

typedef enum {
  DDA_OK = 0,
  DDA_EINVAL = 1,        /* bad argument (shape, size, pointer, enum) */
  DDA_ENOMEM = 2,        /* device or host allocation failed */
  DDA_ECUDA = 3,         /* a CUDA runtime call failed */
  DDA_ENOCONV = 4,       /* solver stopped at maxit without reaching tol */
  DDA_ETIMEOUT = 5,      /* solver exceeded its wall-clock budget */
  DDA_ESTATE = 6,        /* call made before the state it needs */
  DDA_EUNSUPPORTED = 7   /* valid request this build does not implement */
} dda_status;

/* Element types.  DDA_C128DF is not a storage type: products asked for in it
 * read and write complex128 vectors but compute in double-float arithmetic
 * (each FP64 value carried as an unevaluated sum of two floats, 48 significand
 * bits) on the FP32 units, because GB300's FP64 rate is 1/64 of its FP32 rate.
 * Its results agree with the complex128 product to about 1e-13 of the norm of
 * the result; it exists where the complex128 schedule has compile-time kernels
 * (dda_schedule_info(DDA_C128) info[1] = 1 and info[0] = 5), else the calls
 * that take it return DDA_EUNSUPPORTED. */
enum { DDA_C64 = 1, DDA_C128 = 2, DDA_C128DF = 3 };
/* Target shapes (guide, "Target Generation"); SHPAR in lattice units. */
enum { DDA_ELLIPSOID = 1, DDA_RCTGLPRSM = 2, DDA_CYLINDER1 = 3, DDA_HEX_PRISM = 4 };
/* Polarizability prescriptions (guide, "Dipole Polarizabilities"). */
enum { DDA_CM = 1, DDA_LATTDR = 2, DDA_GKDLDR = 3 };
/* Iterative solvers (guide, "Choice of Iterative Algorithm"): BiCGstab (van
 * der Vorst 1992, the guide's PBCGST), CCG (conjugate gradients on the normal
 * equations, Petravic & Kuo-Petravic 1979, the guide's PETRKP) and
 * BiCGstab(2) (Sleijpen & Fokkema 1993, the method family of the guide's
 * recommended PBCGS2, without that routine's reliability refinements). */
enum { DDA_BICGSTAB = 1, DDA_CCG = 2, DDA_BICGSTAB2 = 3, DDA_COCG = 4, DDA_QMRCS = 5 };
/* DDA_COCG: conjugate orthogonal conjugate gradients (van der Vorst & Melissen
 * 1990), CG with the unconjugated form x^T y, valid because A is complex
 * symmetric (A^T = A); one product per iteration (the complex-symmetric
 * Lanczos family of the guide's QMRCCG option).
 * DDA_QMRCS: QMR for complex-symmetric A (Freund 1992, the guide's QMRCCG
 * option), on the symmetric Lanczos process without look-ahead; one product per
 * iteration; stops when sqrt(n + 1) |tau_bar| (its bound on the true residual
 * after n steps) reaches tol |E|; complex128 only (DDA_EUNSUPPORTED for the
 * complex64 and mixed precisions: without look-ahead its Lanczos vectors meet
 * near breakdowns, v^T v ~ 0, that complex64 cannot carry).  Both need A
 * complex symmetric: not for periodic targets at oblique incidence. */
/* Preconditioning of the iterations (guide, "Choice of Iterative Algorithm":
 * the guide's solvers are preconditioned Krylov methods): none, or Jacobi, the
 * diagonal of A, applied symmetrically -- the solver iterates on
 * (S A S) y = S E with S = diag(alpha^{1/2}) and returns P = S y, which keeps
 * the operator complex symmetric for DDA_COCG.  The iterations test the scaled
 * residual |S (E - A P)| / |S E| against tol / kappa, kappa = max |s| / min |s|
 * over the polarizability table, which guarantees |E - A P| / |E| <= tol for
 * the complex64 and complex128 solves (mixed-precision solves test the true
 * residual in their outer loop anyway). */
enum { DDA_PRECOND_NONE = 0, DDA_PRECOND_JACOBI = 1 };
/* Arithmetic of the solve: all complex64, all complex128, or complex64 inner
 * iterations refined against complex128 true residuals. */
enum { DDA_PREC_C64 = 1, DDA_PREC_C128 = 2, DDA_PREC_MIXED = 3 };

/* Create a context on CUDA device `device`, enqueuing on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out receives the
 * context, or NULL on failure (then the message is lost: only the status).
 * device < 0 creates a host-only context: target, incidence and
 * polarizability set-up and their getters work without a GPU; every call that
 * needs the device returns DDA_ESTATE. */
DDA_API dda_status dda_create(dda_ctx **out, int device, void *cuda_stream);
/* Free everything the context owns.  NULL is accepted. */
DDA_API void dda_destroy(dda_ctx *ctx);
/* Message for the last failing call on ctx ("" if none).  Owned by ctx. */
DDA_API const char *dda_last_error(const dda_ctx *ctx);
/* Change the stream later work is enqueued on. */
DDA_API dda_status dda_set_stream(dda_ctx *ctx, void *cuda_stream);

/* Built-in target (guide, "Target Generation": ELLIPSOID, RCTGLPRSM, CYLINDER1,
 * HEX_PRISM).  shpar[0..nshpar) are SHPAR_1.. in lattice units (lengths must
 * be positive integers; CYLINDER1 needs SHPAR_3 in 1..3, HEX_PRISM in 1..6).
 * Sites sit at cell centres, the Target-Frame origin at the centroid
 * (RCTGLPRSM: centre of the upper x face); surface ties count as inside.
 * Outputs: *n_out = number of occupied sites N, box_out = bounding box
 * (Nx, Ny, Nz).  Either output pointer may be NULL.  Replaces any earlier
 * target and drops the incident, Green and polarizability state. */
DDA_API dda_status dda_setup_shape(dda_ctx *ctx, int shape, const double *shpar, int nshpar, int64_t *n_out,
                           int32_t box_out[3]);

/* Target from a site list (the guide's FROM_FILE route): ixyz is host N x 3
 * integer lattice coordinates (any order, no duplicates), icomp host N
 * composition indices (1-based, NULL = all 1), origin_tf the Target-Frame
 * position of lattice point (0,0,0), a1/a2 the target axes in the TF (NULL =
 * x_TF, y_TF).  Sites are re-ordered x-fastest; dda_get_sites reports the order. */
DDA_API dda_status dda_setup_target(dda_ctx *ctx, const int32_t *ixyz, const int32_t *icomp, int64_t n,
                            const double origin_tf[3], const double a1[3], const double a2[3]);

/* The same for a target of anisotropic materials whose principal axes are the
 * Target-Frame axes (the guide's FROM_FILE targets with a composition per
 * site and axis, section "FROM_FILE = Target composed of possibly anisotropic
 * material"): icomp3 host N x 3, the 1-based
 * composition of each site's x, y and z axis; dda_set_polarizability then
 * gives one refractive index per composition, and axis a of a site takes the
 * polarizability of its axis-a composition. */
DDA_API dda_status dda_setup_target_aniso(dda_ctx *ctx, const int32_t *ixyz, const int32_t *icomp3, int64_t n,
                                  const double origin_tf[3], const double a1[3], const double a2[3]);

/* The guide's ANIFRMFIL target (section "ANIFRMFIL = General anisotropic
 * target"; "Composite Targets with Anisotropic Constituents"): like
 * dda_setup_target_aniso, plus df_angles host N x 3 = (theta_DF, phi_DF,
 * beta_DF) in radians, the orientation of each site's Dielectric Frame (the
 * principal axes e_1, e_2, e_3 of its dielectric tensor) relative to the TF by
 * the guide's three rotations; icomp3[j][a] is the composition along e_a.
 * dda_set_polarizability then gives each site the full symmetric tensor
 * alpha^{-1} = sum_a d_a e_a e_a^T, d_a the prescription's alpha^{-1} for the
 * composition of axis a with the incidence (khat, polarization) projected on
 * the principal axes (for zero angles this is exactly dda_setup_target_aniso).
 * Products, solves and efficiencies then use the full tensor; the Jacobi
 * preconditioner returns DDA_EUNSUPPORTED and true residuals use the complex128
 * product (no DDA_C128DF) for such targets. */
DDA_API dda_status dda_setup_target_anifrm(dda_ctx *ctx, const int32_t *ixyz, const int32_t *icomp3, int64_t n,
                                           const double origin_tf[3], const double a1[3], const double a2[3],
                                           const double *df_angles);

/* Copy the site list out (guide, "Target Generation: Isolated Finite Targets": the
 * dipole sites of the target on the lattice): ixyz_out host N x 3 (box-relative lattice indices),
 * origin_out[3] = TF position of box index (0,0,0).  Either may be NULL. */
DDA_API dda_status dda_get_sites(dda_ctx *ctx, int32_t *ixyz_out, double origin_out[3]);

/* The current target's site count and bounding box (cells per axis, x y z), as
 * dda_setup_shape reports them; n_out and box_out may be NULL.  DDA_ESTATE
 * without a target (the context is const: no dda_last_error message). */
DDA_API dda_status dda_get_box(const dda_ctx *ctx, int64_t *n_out, int32_t box_out[3]);

/* Periodic targets (guide, "Target Generation: Periodic Targets" and
 * "Interaction Cutoff Parameter for PBC Calculations"; Draine & Flatau 2008):
 * the current target becomes the Target Unit Cell, repeated with period py
 * along y_TF and / or pz along z_TF (lattice units; 0 = no repetition along
 * that axis; a nonzero period must be at least the cell's extent).  Under the
 * incident wave of TF wave vector k the replica displaced by R carries the
 * cell's polarization times exp(i k.R), and the product becomes
 * alpha^{-1} P + sum_k A^per(r_j - r_k) P_k with A^per(r) = sum_R exp(i k.R)
 * A(r - R) exp[-(gamma kd |r - R|)^4] (the term r - R = 0 omitted; replicas
 * kept while (gamma kd |r - R|)^4 <= 40), built in FP64 by
 * dda_build_green_fft on the full wrapped grid (O(grid points x replicas)).
 * Every RHS of the context must then share one incident direction in the TF
 * (one orientation, or orientations differing only in Phi), else
 * dda_build_green_fft returns DDA_EUNSUPPORTED.  Efficiencies from
 * dda_cross_sections are per unit cell (a_eff of the cell); Mueller matrices,
 * angular averages, force and torque and near fields return
 * DDA_EUNSUPPORTED for periodic targets.  gamma in (0, 1) (the guide suggests
 * 1e-2, smaller for accuracy).  Call after the target; py = pz = 0 makes the
 * target finite again.  Drops the Green tensor. */
DDA_API dda_status dda_set_periodicity(dda_ctx *ctx, double py, double pz, double gamma);

/* Lattice wavenumber for a size parameter (guide, "Target Generation" and the
 * definitions of a_eff and x): the target's effective radius is
 * a_eff = (3 N / 4 pi)^(1/3) d, the radius of a sphere of volume N d^3, and
 * x = k a_eff, so kd = x / (a_eff / d).  x > 0.  Outputs (either may be NULL):
 * *kd_out = kd, *aeff_out = a_eff / d.  DDA_ESTATE without a target, DDA_EINVAL for
 * x <= 0 or a non-finite x (the context is const: these two set no dda_last_error
 * message).  Host only; pass kd to dda_set_incident. */
DDA_API dda_status dda_kd_from_x(const dda_ctx *ctx, double x, double *kd_out, double *aeff_out);

/* Incident beams (guide, "Target Orientation" and "Incident Polarization
 * State").  kd = k d (lattice wavenumber, > 0).  ori: host n_ori x 3 angles
 * (beta, Theta, Phi) in radians.  e01_lf: host 6 doubles, the Lab-Frame
 * components (x, y, z) of e01 as (re, im) pairs; normalized here.  iorth = 1
 * (e01 only) or 2 (adds e02 = x_LF x e01*).  Defines nrhs = n_ori * iorth
 * right-hand sides, index = ori * iorth + pol. */
DDA_API dda_status dda_set_incident(dda_ctx *ctx, double kd, const double *ori, int n_ori, const double e01_lf[6],
                            int iorth);

/* Number of right-hand sides defined by dda_set_incident (0 before). */
DDA_API int dda_nrhs(const dda_ctx *ctx);

/* Copy the incidence out (guide, "Orientation of the Incident Beam in the Target
 * Frame" and "Incident Polarization State"): k_tf host nrhs x 3 (k vector in the Target Frame,
 * lattice units), e_tf host nrhs x 6 (polarization in the TF, (re, im) x 3).
 * Either may be NULL. */
DDA_API dda_status dda_get_incidence(dda_ctx *ctx, double *k_tf, double *e_tf);

/* Write the incident plane wave at the sites (the right-hand side E of the guide's
 * A P = E, "Choice of Iterative Algorithm"; beam and polarization from "Orientation of
 * the Incident Beam in the Target Frame" and "Incident Polarization State"):
 * E_inc,j = e exp(i k . r_j) for every RHS into e_dev ([nrhs][3][N],
 * dtype DDA_C64 or DDA_C128), phases evaluated in FP64. */
DDA_API dda_status dda_incident_field(dda_ctx *ctx, void *e_dev, int dtype);

/* Dipole-dipole tensor on the padded FFT grid and its FFT (Goodman, Draine &
 * Flatau 1991), filled and transformed in FP64 on the device and kept in
 * complex128 and rounded complex64 copies.  pad = padded grid (Px, Py, Pz),
 * each even, >= 2 N_axis and a product of 2, 3 and 5; NULL = the smallest
 * such lengths (the guide's extended computational volume).  Uses the kd
 * given to dda_set_incident.  Also picks the launch schedule of the product
 * for this grid (3-pass when a y-z plane fits in shared memory, else 5-pass). */
DDA_API dda_status dda_build_green_fft(dda_ctx *ctx, const int32_t pad[3]);

/* Polarizabilities (guide, "Dipole Polarizabilities"), after dda_set_incident: prescription DDA_CM
 * (Clausius-Mossotti with radiative reaction), DDA_LATTDR (Draine & Goodman
 * 1993) or DDA_GKDLDR (Gutkowicz-Krusin & Draine 2004).  m_reim: host ncomp x 2
 * refractive indices relative to the medium, one per composition.  Computed
 * per RHS (they depend on the incidence) in FP64. */
DDA_API dda_status dda_set_polarizability(dda_ctx *ctx, int prescription, const double *m_reim, int ncomp);

/* Copy the diagonal of alpha^{-1} out (guide, "Dipole Polarizabilities": the diagonal
 * blocks of A): host nrhs x ncomp x 3 complex (re, im). */
DDA_API dda_status dda_get_inv_alpha(dda_ctx *ctx, double *out);

/* The product with the DDA matrix (guide, eq. AP=E in "Choice of Iterative Algorithm";
 * the off-diagonal part as the FFT convolution of "Choice of FFT Algorithm"):
 * ap_dev = A p_dev for the first nrhs right-hand sides, both [nrhs][3][N] of
 * dtype DDA_C64 or DDA_C128 (may not alias); DDA_C128DF takes and returns
 * complex128 vectors and computes in double-float arithmetic.  Enqueue only. */
DDA_API dda_status dda_matvec(dda_ctx *ctx, const void *p_dev, void *ap_dev, int nrhs, int dtype);

/* ap_dev = A p_dev like dda_matvec, but without allocating any memory.
 * The guide has no counterpart: this entry point exists for callers that
 * cannot allocate device memory -- for example code whose device memory is
 * owned by another allocator under a fixed budget (a framework's caching
 * pool), or latency-sensitive loops where cudaMalloc/cudaFree would
 * synchronize the device and stall other streams.  Instead of the context's
 * grown-on-demand workspace, the product's FFT scratch lives in one fixed
 * array of 32 MiB inside the library's device image; every GPU that loads the
 * library holds those 32 MiB until the process exits.  Requests whose scratch
 * (sizeof(complex) x 3 x Px x Nz x Ys per RHS, Ys = Ny on the 3-pass schedule,
 * Py on the 5-pass one) exceeds 32 MiB return DDA_EINVAL with the sizes in the
 * message.  The call makes no cudaMalloc, cudaFree or other allocating call.
 * The array's device address is looked up once per device, with that device
 * current, by the first dda_build_green_fft on the device (a prerequisite of
 * this call; the array sits in the same device module as the Green-tensor
 * kernels that call has just run, so the lookup loads nothing new); this call
 * then only reads the cached address.  Do not reset the device
 * (cudaDeviceReset) between dda_build_green_fft and this call: a reset unloads
 * the module and the cached address would be stale.  Every call shares the one
 * array and it keeps the last call's contents; nothing in it has to start at
 * zero because each pass writes all the scratch the next pass reads.  Calls
 * whose work overlaps on the GPU (other streams, other threads, other contexts
 * on the same device) race on the array: serialize them.  The context must
 * already hold the Green tensor and the polarizabilities (both allocated
 * earlier by their own calls).  The product uses the context's schedule, except
 * that it stages the plane pass with bulk copies only when the context already
 * has its fault flag (made by an earlier dda_matvec or dda_solve): a bounded
 * bulk-copy wait that gives up is reported only through that flag, by the next
 * synchronizing call (dda_solve, dda_profile_matvec) as DDA_ECUDA.  Enqueue only. */
DDA_API dda_status dda_matvec_noalloc(dda_ctx *ctx, const void *p_dev, void *ap_dev, int nrhs, int dtype);

typedef struct {
  int solver;        /* DDA_BICGSTAB, DDA_CCG, DDA_BICGSTAB2, DDA_COCG or DDA_QMRCS */
  int precision;     /* DDA_PREC_C64 / DDA_PREC_C128 / DDA_PREC_MIXED */
  double tol;        /* stop when |E - A P| / |E| <= tol for every RHS */
  int maxit;         /* iteration cap (inner iterations summed for MIXED) */
  double inner_tol;  /* MIXED: smallest relative reduction asked of an inner complex64 solve; each
                        inner solve aims at 0.8 tol / (current true relative residual) but not
                        below this floor (0 = 5e-6, near the complex64 limit) */
  double timeout_ms; /* wall-clock budget, 0 = none; exceeded -> DDA_ETIMEOUT */
  int warm_start;    /* 1 = p_dev holds the initial guess, 0 = start from P = 0 */
  int check_every;   /* iterations between host convergence checks (0 = 8; BiCGstab(2): cycles of two iterations) */
  int normal_eq;     /* 1 = also evaluate the guide's normal-equation ratio at exit (2 extra FP64 products) */
  int use_graph;     /* 1 = replay the iterations as a captured CUDA graph, 0 = plain launches */
  int precond;       /* DDA_PRECOND_NONE or DDA_PRECOND_JACOBI */
  int phi_reuse;     /* 1 = orientations that differ from an earlier one only in Phi are not iterated
                        on: with iorth = 2 and a polarizability that does not depend on the incident
                        polarization (DDA_CM, DDA_GKDLDR), their solutions are linear combinations of
                        the earlier orientation's two (guide, note on IPHI > 1 in "Scattering
                        Amplitude Matrix"); ignored otherwise.  Their reports show 0 iterations and
                        their own FP64 true residual. */
} dda_solve_opts;

typedef struct {
  int iters;             /* Krylov iterations used (inner ones for MIXED) */
  int matvecs;           /* products with A applied to this RHS (any precision; a batch skips the
                            products of RHS whose solve has finished) */
  int outer;             /* MIXED: refinement steps (true-residual evaluations) */
  int converged;         /* 1 if the true residual met tol */
  double true_rel_resid; /* |E - A P| / |E| evaluated with an FP64-accurate product at exit: the
                            complex128 product, or for precisions C64 and MIXED at tol >= 1e-10 the
                            double-float one (DDA_C128DF) where it exists (environment variable
                            DDA_RESIDUAL=fp64 forces the complex128 product) */
  double normal_eq_ratio;/* guide's eq. err_tol: |A^H A P - A^H E| / |A^H E| (NAN if not computed) */
} dda_solve_report;

/* Solve A P = E_inc for every RHS (guide, "Choice of Iterative Algorithm"; stopping
 * rule: the true relative residual, with the guide's normal-equation ratio of "Error
 * Tolerance" reported on request).  p_dev: [nrhs][3][N] complex128 (always
 * FP64 storage), initial guess when opt->warm_start, solution on return.
 * rep: host array of nrhs reports (may be NULL).  Returns DDA_ENOCONV if any
 * RHS missed tol within maxit (p_dev and rep still hold the last iterate). */
DDA_API dda_status dda_solve(dda_ctx *ctx, const dda_solve_opts *opt, void *p_dev, dda_solve_report *rep);

/* Solve several targets at once (the guide runs independent problems as separate
 * processes, "MPI: Message Passing Interface"; here they share one device), for mixed
 * batches: targets of uneven grid sizes
 * on one device).  ctxs[i] are distinct contexts on the same
 * device, each fully set up (target, incidence, Green tensor, alpha) with its
 * own product schedule; p_devs[i] their complex128 [nrhs_i][3][N_i] buffers;
 * reps[i] host arrays of nrhs_i reports (or reps = NULL); statuses host array
 * of nctx statuses (or NULL).  Every target runs the same algorithm as
 * dda_solve, each replaying its iterations as its own CUDA graph on its own
 * stream from its own host thread, so the targets' kernels share the GPU
 * concurrently and small targets fill SMs that one target alone leaves idle.
 * Product schedules are autotuned one target at a time before the concurrent
 * part starts, so the tuner's timings are not disturbed by the other targets.
 * Returns DDA_OK if every target succeeded, else the first failing status.
 * Returns after all targets finished. */
DDA_API dda_status dda_solve_batch(dda_ctx *const *ctxs, int nctx, const dda_solve_opts *opt, void *const *p_devs,
                                   dda_solve_report *const *reps, dda_status *statuses);

/* Scattering of a periodic target (dda_set_periodicity) into its allowed
 * directions, for a solved P (complex128 [nrhs][3][N], device) (guide,
 * "Scattering Directions for Targets that are Periodic in 1 Dimension", "...
 * for Doubly-Periodic Targets" and "Scattering by Periodic Targets:
 * Generalized Mueller Matrix").  spec: host n_spec x 2 doubles.  Doubly
 * periodic: the diffraction orders (M, N) (integers); the order's direction
 * has k_y = k0_y + 2 pi M / P_y, k_z = k0_z + 2 pi N / P_z and |k_x| fixed by
 * |k| = k0, on the transmission (sign of k0_x) and the reflection side.
 * Singly periodic: (M, zeta), cone order M along the repetition axis and
 * azimuth zeta (radians): axis y -> (k_perp cos zeta, k_y, k_perp sin zeta),
 * axis z -> (k_perp cos zeta, k_perp sin zeta, k_z).  Outputs (host, each may
 * be NULL):
 *   dirs_out    n_spec x 2 x 3: TF unit vectors (transmission, reflection;
 *               singly periodic: the cone direction, then zeros);
 *   mueller_out n_ori x n_spec x 2 x 16 (row-major; needs iorth = 2): the
 *               guide's generalized Mueller matrix, I_sca = S^(2d) I_in for
 *               the plane wave of order (M, N) (transmission then reflection),
 *               I_sca = S^(1d) I_in / (k rho) at distance rho from the axis
 *               (slot 1 zero); the incident wave is not part of the scattered
 *               Stokes vector;
 *   tr_out      nrhs x n_spec x 2 (doubly periodic only): fractions of the
 *               incident power per unit area carried by the order in
 *               transmission (including the incident wave for (0, 0)) and in
 *               reflection; with the absorbed fraction they sum to 1 over the
 *               allowed orders.
 * Normalisation read from the replicas' plane-wave (Weyl) and cylindrical-wave
 * sums: S^(2d) = S(n) (2 pi / (A k k_x))^2, S^(1d) = S(n) 2 pi / (k k_perp L^2),
 * S(n) the finite-target Mueller matrix of the same P in direction n, A the
 * cell area.  DDA_EINVAL for an order that does not propagate (the guide's
 * condition on M, N) or a non-integer order; DDA_EUNSUPPORTED for a finite
 * target.  Synchronizes the stream. */
DDA_API dda_status dda_periodic_scattering(dda_ctx *ctx, const void *p_dev, int n_spec, const double *spec,
                                           double *dirs_out, double *mueller_out, double *tr_out);

/* Efficiencies and Mueller matrices for a solved P (complex128 [nrhs][3][N]).
 * q_out: host nrhs x 4 doubles (Q_ext, Q_abs, Q_sca = Q_ext - Q_abs, Q_pha),
 * Q = C / (pi a_eff^2), formulas of Draine 1988 as used by the guide.
 * dirs: host ndir x 2 (theta_s, phi_s) radians in the Lab Frame (guide,
 * CMDFRM = LFRAME); mueller_out: host n_ori x ndir x 16 doubles (row-major S_ij,
 * guide's Mueller relations) -- needs iorth = 2; pass ndir = 0 / NULL to skip.
 * Synchronizes the stream. */
DDA_API dda_status dda_cross_sections(dda_ctx *ctx, const void *p_dev, double *q_out, const double *dirs, int ndir,
                              double *mueller_out);

/* Number of CUDA kernels the library has launched in this process (graph
 * replays counted node by node).  For accounting in benchmarks. */
DDA_API unsigned long long dda_kernel_launches(void);

/* Time the product's passes: runs `iters` products A p (p = 0, scratch
 * buffers owned by the call) for nrhs RHS in dtype, with CUDA events recorded
 * on the context's stream between the passes, and writes the mean duration of
 * each pass in ms to ms_per_pass (up to 5 entries; *npass receives 3 for the
 * 3-pass schedule: x forward, fused y-z plane, x inverse; or 5 for the 5-pass
 * schedule: x forward, y forward, z, y inverse, x inverse).  Synchronizes. */
DDA_API dda_status dda_profile_matvec(dda_ctx *ctx, int nrhs, int dtype, int iters, double *ms_per_pass, int *npass);

/* Launch schedule of the product for dtype, as chosen by the autotuner (the
 * first product for a given RHS count times the candidate schedules and keeps
 * the fastest) or pinned by the DDA_SCHEDULE environment variable at
 * dda_build_green_fft time ("generic", "fast5", "plane512", "plane768",
 * "cluster2", "cluster4"; DDA_XTILE = 4, 8 or 16 pins the x passes' tile
 * height; DDA_BULK = 1 or 0 pins bulk-copy staging of the plane pass;
 * DDA_XCOMP = 1 runs the x passes with one field component per CTA).
 * info[0] = passes (3 = fused y-z plane, 5 = split), info[1] = 1 when the
 * compile-time-length kernels are used, info[2] = threads per CTA of the plane
 * kernel (0 if none), info[3] = RHS count the choice was tuned for (0 = not
 * tuned), info[4] = CTAs per plane (1, or the thread-block cluster size when
 * the plane pass is split over a cluster), info[5] = y rows per CTA of the x
 * passes (0 for the generic engine), info[6] = 1 when the plane pass stages its
 * HBM blocks with bulk copies (TMA), info[7] = field components per CTA of the
 * x passes (3 or 1; 0 for the generic engine), info[8] = 1 when the 5-pass z
 * columns run pass B, the Ghat multiply and the inverse pass B of the three
 * components in registers (a tuner candidate for long z transforms); info[9..11]
 * are reserved (0). */
DDA_API dda_status dda_schedule_info(dda_ctx *ctx, int dtype, int32_t info[12]);

/* ---------------------------------------------------------------------------
 * Learned warm start (the guide has no counterpart: the solver accepts any
 * initial guess, and a network trained on the solver's own solutions gives a
 * better one).  A small 3-D U-Net maps per-voxel features of a target on a grid
 * of dims (x, y, z), each a multiple of 8 covering the box, to the local field
 * E_loc = alpha^{-1} P; the warm start is P0 = alpha E_loc.  Tensors are FP32,
 * channels-last [batch][z][y][x][channel], on the device.
 * ------------------------------------------------------------------------- */
typedef struct dda_unet dda_unet;

/* Network with cin input and cout output channels and level widths ch[0..3]
 * (each 1..64), He-uniform weights from seed; work on `cuda_stream`.  The
 * 3x3x3 convolutions (forward and input gradient) run as implicit GEMMs on the
 * tensor cores: tcgen05 MMAs with tensor-memory accumulators on halo tiles
 * staged by TMA from a bfloat16 copy of the input (rows of at most 254 voxels;
 * longer rows use mma.sync), or mma.sync throughout when the environment
 * variable DDA_UNET_TC=0 is set at creation.  The tcgen05 kernel's mbarrier
 * waits are bounded; a wait that gives up is reported by dda_unet_check_fault.
 * The 1x1x1 head and the weight gradients use mma.sync in both modes. */
DDA_API dda_status dda_unet_create(dda_unet **out, int device, void *cuda_stream, int cin, int cout, const int32_t ch[4],
                                   uint64_t seed);
DDA_API void dda_unet_destroy(dda_unet *net);
/* DDA_ECUDA if a tcgen05 convolution's bounded completion wait gave up since the
 * last call (its outputs are then invalid; the flag is cleared), else DDA_OK.
 * Call after synchronizing the network's stream; dda_unet_loss_grad makes this
 * check itself before it returns. */
DDA_API dda_status dda_unet_check_fault(dda_unet *net);
DDA_API const char *dda_unet_last_error(const dda_unet *net);
DDA_API int64_t dda_unet_nparams(const dda_unet *net);
/* Copy the FP32 parameters (which = 0) or their last gradients (which = 1) to
 * host memory, layer by layer W[tap][cin][cout] then b.  Synchronizes. */
DDA_API dda_status dda_unet_get_params(dda_unet *net, float *host, int which);
DDA_API dda_status dda_unet_set_params(dda_unet *net, const float *host);
/* y = net(x) for `batch` grids of the given dims. */
DDA_API dda_status dda_unet_forward(dda_unet *net, const float *x_dev, float *y_dev, int batch, const int32_t dims[3]);
/* Masked mean-squared error against t (mask [batch][z][y][x] of 0/1) and its
 * gradient w.r.t. every parameter (kept in the network for dda_unet_adamw);
 * *loss_out receives the loss.  Synchronizes. */
DDA_API dda_status dda_unet_loss_grad(dda_unet *net, const float *x_dev, const float *t_dev, const float *mask_dev,
                                      int batch, const int32_t dims[3], double *loss_out);
/* Training with an arbitrary loss: forward pass keeping the activations for
 * dda_unet_backward (same batch and dims), weight times the masked
 * mean-squared error's value and gradient gy_dev = dL/dy (overwritten), and
 * the backward pass from a given dL/dy (gradients kept for dda_unet_adamw).
 * Synchronizing calls: dda_unet_mse. */
DDA_API dda_status dda_unet_forward_train(dda_unet *net, const float *x_dev, float *y_dev, int batch,
                                          const int32_t dims[3]);
DDA_API dda_status dda_unet_mse(dda_unet *net, const float *y_dev, const float *t_dev, const float *mask_dev,
                                int batch, const int32_t dims[3], double weight, float *gy_dev, double *loss_out);
DDA_API dda_status dda_unet_backward(dda_unet *net, const float *gy_dev, int batch, const int32_t dims[3]);
/* One AdamW step (decoupled weight decay wd) with the stored gradients. */
DDA_API dda_status dda_unet_adamw(dda_unet *net, double lr, double beta1, double beta2, double eps, double wd);
/* Features of every RHS of ctx on the grid: x_dev [nrhs][z][y][x][9] =
 * [occupied, (Re eps - 1)/4, Im eps / 2, Re/Im of E_inc x, y, z], zero outside
 * the target.  offset = position of box index (0,0,0) in the grid (NULL = centred). */
DDA_API dda_status dda_unet_features(dda_ctx *ctx, float *x_dev, const int32_t dims[3], const int32_t offset[3]);
/* Training targets from a solution p_dev (complex128 [nrhs][3][N]):
 * t_dev [nrhs][z][y][x][6] = Re/Im of alpha^{-1} P (residual = 0) or of
 * alpha^{-1} P - E_inc (residual = 1: the network learns the correction to the
 * local field being the incident field), mask_dev [nrhs][z][y][x]. */
DDA_API dda_status dda_unet_targets(dda_ctx *ctx, const void *p_dev, float *t_dev, float *mask_dev,
                                    const int32_t dims[3], const int32_t offset[3], int residual);
/* Initial guess p_dev (complex128 [nrhs][3][N]) = alpha * E_loc from network
 * output y_dev [nrhs][z][y][x][6], E_loc = y (+ E_inc when residual = 1); pass
 * it to dda_solve with warm_start = 1. */
DDA_API dda_status dda_unet_warm_start(dda_ctx *ctx, const float *y_dev, const int32_t dims[3],
                                       const int32_t offset[3], int residual, void *p_dev);

/* Residual loss of a network output for ctx: with P0 = alpha (E_inc + y)
 * (residual-mode output y_dev [nrhs][z][y][x][6] on the grid), adds
 * weight * sum_b |E_b - A P0_b|^2 / |E_b|^2 to *loss_out and its gradient to
 * gy_dev (same layout, accumulated), computed with the complex64 product and
 * its adjoint A^H x = conj(A conj x).  This trains the network on the quantity
 * the solver's convergence depends on.  Synchronizes. */
DDA_API dda_status dda_unet_residual_grad(dda_ctx *ctx, const float *y_dev, const int32_t dims[3],
                                          const int32_t offset[3], double weight, float *gy_dev, double *loss_out);

/* Angular averages over scattering directions (guide, "Averaging over
 * Scattering Directions"): the guide's direction set for x = k a_eff and eta
 * (theta_j equally spaced in s(theta) = theta + theta/(theta + theta0),
 * theta0 = 2 pi/(1 + x), N_theta = nint of the guide's expression in eta,
 * N_phi(j) = max(3, nint(4 pi sin theta_j / (theta_{j+1} - theta_{j-1}))),
 * phi_{j,k} = 2 pi (k-1)/N_phi(j), solid-angle weights Omega_{j,k}), applied to
 * dC_sca/dOmega = k^4 |F - n (n . F)|^2 with F = sum_j P_j exp(-i k n . r_j).
 * p_dev: the solved P (complex128 [nrhs][3][N], device).  out[nrhs][6] =
 * Q_sca by integration, <cos theta>, <cos^2 theta>, and the Lab-Frame
 * components of <n> (the guide's g vector), all intensity-weighted.
 * *ndir_out = number of directions (the guide's N_sca).  The far-field sums
 * run on the device with FP32 phases from FP64 separable tables and FP64
 * block totals.  Synchronizes. */
DDA_API dda_status dda_angular_averages(dda_ctx *ctx, const void *p_dev, double eta, double *out,
                                        int32_t *ndir_out);

/* Radiative force and torque efficiency vectors (guide, "Calculation of
 * <cos theta>, Radiative Force, and Radiation Torque"): Q_pr = F_rad /
 * (pi a_eff^2 u_rad) and Q_Gamma = k Gamma_rad / (pi a_eff^2 u_rad), u_rad =
 * |E0|^2 / 8 pi, for a solved P (complex128 [nrhs][3][N], device).  The force
 * is Q_ext khat - Q_sca g; the torque (about the centroid of the sites) is the
 * incident field's torque on the dipoles, sum_j [1/2 Re(P_j x E_inc,j^*) +
 * (k/2) Im(P_j . E_inc,j^*) r_j x khat], plus the torque of the array's own
 * radiative field, (k^3/8pi) oint Im[g x f^*] - (k^4/8pi) oint Re[h] x n with
 * g = sum_j P_j exp(-i k n.r_j), f = g - n (n.g), h = T f^*, T[c][a] =
 * sum_j r_jc P_ja exp(-i k n.r_j), integrated over the guide's scattering
 * directions for eta (as dda_angular_averages; the guide notes that both
 * vectors need an adequate ETASCA).  out: host nrhs x 6 = Q_pr then Q_Gamma,
 * Target-Frame components.  *ndir_out (may be NULL) = directions used.
 * Far-field sums in FP32 from FP64 phase tables, totals in FP64.  Synchronizes. */
DDA_API dda_status dda_force_torque(dda_ctx *ctx, const void *p_dev, double eta, double *out, int32_t *ndir_out);

/* Electric and magnetic fields in or near the target (guide, "Postprocessing:
 * Calculating E and B In or Near the Target", the DDfield program) for a
 * solved P (complex128 [nrhs][3][N], device): at each point x (host npts x 3,
 * Target-Frame coordinates in lattice units) E = E_inc + sum_j phi(R_j)
 * E_dip and B = B_inc + sum_j phi(R_j) B_dip, the retarded fields of the
 * oscillating point dipoles P_j at distance R_j = |x - r_j|, with the incident
 * plane wave E_inc = e exp(i k.x), B_inc = khat x E_inc (Gaussian units, time
 * factor exp(-i w t) = 1).  The contribution of dipoles closer than one lattice
 * spacing is suppressed by phi(R) = R^4 (5 - 4 R) (R < 1; phi = 1 beyond), a
 * factor vanishing faster than R^3 as the guide asks.  e_out / b_out: host
 * [nrhs][npts][6] = (re, im) of x, y, z; b_out may be NULL.  Direct FP64 sum
 * over all dipoles on the device (O(N npts)).  Periodic targets
 * (dda_set_periodicity): the sum runs over the replicas R of the unit cell too,
 * moments P_j exp(i k.R), each term also weighted by the interaction cutoff
 * exp[-(gamma k D)^4] of its distance D and dropped where (gamma k D)^4 > 40
 * (O(N npts replicas); DDA_EINVAL beyond 2e11 terms).  Synchronizes. */
DDA_API dda_status dda_near_field(dda_ctx *ctx, const void *p_dev, const double *pts, int64_t npts, double *e_out,
                                  double *b_out);

/* Orientation grid for orientational averaging (guide, "Sampling in Theta,
 * Phi, and beta" and "Orientational Averaging"): beta and Phi at the midpoints
 * of nbeta / nphi equal intervals of [min, max] (degrees); cos(Theta) uniform:
 * ntheta odd -> the end points included with Simpson weights
 * (1/3, 4/3, 2/3, ..., 4/3, 1/3)/(ntheta - 1), ntheta even -> interval
 * midpoints with equal weights.  ori_out [nbeta*ntheta*nphi][3] = (beta,
 * Theta, Phi) in radians, Phi fastest then Theta then beta (pass it to
 * dda_set_incident); w_out [n] = weights (they sum to one; the average of a
 * quantity over orientations is sum_o w_o Q_o).  Host only. */
DDA_API dda_status dda_orientation_grid(const double beta_deg[2], int nbeta, const double theta_deg[2], int ntheta,
                                        const double phi_deg[2], int nphi, double *ori_out, double *w_out);

/* Orientational average (guide, "Orientational Averaging"): the weighted sum
 * over orientations <Q> = sum_o w_o Q_o, taken separately for each incident
 * polarization.  w: host n_ori weights (from dda_orientation_grid, or any);
 * vals: host [n_ori][iorth][nval] per-RHS results in the RHS order of
 * dda_set_incident (e.g. the q_out rows of dda_cross_sections: nval = 4 with
 * iorth = 2; Mueller matrices of dda_cross_sections: iorth = 1, nval = ndir x 16);
 * out: host [iorth][nval].  FP64, summed in orientation order.  Host only. */
DDA_API dda_status dda_orientation_average(const double *w, int n_ori, int iorth, const double *vals, int64_t nval,
                                           double *out);

/* Diagnostic (no counterpart in the guide): the product kernels stage their
 * shared-memory blocks with bulk asynchronous copies whose completion waits are
 * bounded; a kernel that gives up records a flag, and the next synchronizing
 * call (dda_solve, dda_profile_matvec) returns DDA_ECUDA.  This call runs that
 * bounded wait on a barrier that never completes, on `device`, and sets
 * *gave_up = 1 when the wait ended by itself (the device stays usable). */
DDA_API dda_status dda_selftest_bulk_wait(int device, int32_t *gave_up);

/* Measurement probe (no counterpart in the guide): applies `reps` unitary
 * 8-point DFT stages to nvec (a multiple of 8) seeded complex vectors held in
 * registers, once with the product's FP32 radix-8 butterflies and once as
 * split-TF32 tensor-core matrix products (mma.sync m16n8k8, three products per
 * stage for an FP32-like error, warp shuffles between stages), on `device`.
 * out[0], out[1] = milliseconds (CUDA events), out[2], out[3] = relative L2
 * error against FP64 of the FP32 and the tensor-core paths.  Allocates and frees
 * its own buffer.  Synchronizes. */
DDA_API dda_status dda_probe_tc_dft(int device, int64_t nvec, int reps, double out[4]);

/* Library build string (static storage). */
DDA_API const char *dda_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DDA_GB300_H */
