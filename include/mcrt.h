/*
 * mcrt.h -- C ABI of the GB300 (sm_103a) library for Monte Carlo dust radiative transfer in
 * optically thick axisymmetric disks, after Min, Dullemond, Dominik, de Koter & Hovenier 2009,
 * "Radiative transfer in very optically thick circumstellar disks" (A&A 497, 155).
 *
 * The library runs three steps on one GPU:
 *   1. Monte Carlo transport of photon packets with immediate (Bjorkman & Wood 2001) re-emission
 *      and the modified random walk (MRW) (Sect. 2.1, 2.2.2, Eq. 5-11)        -> mcrt_run_photons
 *   2. radiative-equilibrium temperatures from the absorbed-energy tallies (Sect. 2.1)
 *                                                                              -> mcrt_temperatures
 *   3. the partial diffusion approximation (PDA), div(D grad T^4) = 0 in the cells that few
 *      packets reached, Monte Carlo temperatures as boundary values (Sect. 2.2.1, Eq. 4)
 *                                                                              -> mcrt_solve_pda
 * plus the escaping-packet spectrum (mcrt_sed) and the adjoint of the PDA solve (mcrt_pda_adjoint);
 * batches of disks in one launch (mcrt_batch_*), the vertical hydrostatic structure (Sect. 2.5, Eq. 20:
 * mcrt_hydrostatic_density), internal sources such as viscous heating (Sect. 5: mcrt_set_sources),
 * polarized transport with a Mueller matrix (Sect. 2.3: mcrt_set_mueller, mcrt_sed_stokes) and
 * ray-traced observables (Sect. 2.3, 4.1: mcrt_set_rays, mcrt_raytrace, mcrt_visibilities) with the
 * scattered light of a mean-intensity tally (mcrt_keep_mean_intensity, mcrt_mean_intensity).
 *
 * Conventions
 *  - Units are cgs at this boundary: cm, g cm^-3, cm^2 g^-1, K, erg s^-1; wavelengths in micron.
 *  - Grid: spherical (r, theta) cells, axisymmetric. Cell (ir, it) spans [r_ir, r_ir+1] x
 *    [theta_it, theta_it+1]; per-cell arrays are row-major [ir * ntheta + it].
 *  - Every call returns an mcrt_status and never aborts or throws across the ABI. On failure the
 *    message is available from mcrt_last_error.
 *  - Inputs are copied by the library; the caller keeps ownership of every pointer it passes.
 *    Host output buffers are caller-owned and filled before the call returns.
 *  - A disk owns its device memory and a CUDA stream (the caller's, when one is given). Calls on
 *    one disk are not thread-safe; distinct disks are independent.
 *  - Functions named *_dev take device pointers and are asynchronous on the disk's stream.
 */
#ifndef MCRT_H
#define MCRT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mcrt_disk mcrt_disk; /* opaque, owned by the library */

typedef enum {
  MCRT_OK = 0,
  MCRT_EINVAL = 1,    /* bad argument: sizes, NaN/negative inputs, unsorted faces, singular PDA region */
  MCRT_ENOMEM = 2,    /* device or host allocation failed */
  MCRT_ECUDA = 3,     /* a CUDA runtime call failed */
  MCRT_ENOTCONV = 4,  /* the PDA solve did not reach its tolerance within its iteration limits */
  MCRT_ETIMEOUT = 5,  /* a device loop hit its iteration guard */
  MCRT_EOVERFLOW = 6, /* a 64-bit fixed-point tally may have wrapped: the energy held by all tallies
                         together (an upper bound of each) passed 2^64 (results invalid) */
  MCRT_ESTATE = 7     /* call order: e.g. transport before mcrt_set_opacity */
} mcrt_status;

/* Fixed-point energy unit: one packet energy (L_star plus any internal sources) / N is 2^16 counts in
 * the 64-bit tallies. */
#define MCRT_EUNIT 65536
/* Inclination bins of the escape spectrum, uniform in |cos i| over [0, 1]. */
#define MCRT_NINC 10

/* Blackbody point star at the origin (Sect. 2.4, Table 1 gives T and R). */
typedef struct {
  double T_star_K;
  double R_star_cm;
} mcrt_star;

/* Grid and dust density (Sect. 2.4, Eq. 17). r_faces_cm: nr+1 increasing radii, r_faces_cm[0] > 0
 * (the region inside is an empty cavity around the star). theta_faces: ntheta+1 increasing polar
 * angles from 0 to pi. rho_gcm3: nr*ntheta densities >= 0. */
typedef struct {
  int nr, ntheta;
  const double *r_faces_cm;
  const double *theta_faces;
  const double *rho_gcm3;
} mcrt_grid;

/* Creates a disk on CUDA device `device`. cuda_stream: a cudaStream_t to run on, or NULL for a
 * stream owned by the disk. *out is set only on success. */
mcrt_status mcrt_disk_create(const mcrt_grid *grid, const mcrt_star *star, int device, void *cuda_stream,
                             mcrt_disk **out);

/* Dust opacities per wavelength bin (Sect. 2.2.1, 2.2.3). lam_edges_um: nlam+1 increasing bin edges.
 * For emission the first bin extends to lambda -> 0 and the last to lambda -> infinity, so the bins
 * hold the whole Planck spectrum. kappa_abs, kappa_sca: mass absorption and scattering coefficients
 * (cm^2/g, kappa_abs > 0). g: Henyey-Greenstein asymmetry per bin, or NULL for isotropic scattering.
 * Identical values in every bin select the gray fast path. Resets the tallies. 1 <= nlam <= 1024. */
mcrt_status mcrt_set_opacity(mcrt_disk *d, int nlam, const double *lam_edges_um, const double *kappa_abs,
                             const double *kappa_sca, const double *g);

/* Packets in flight with non-gray dust. The Bjorkman-Wood re-emission (Sect. 2.1) draws a packet's new
 * wavelength from the temperatures of the moment, and with non-gray dust the wavelength steers the packet.
 * The temperatures then telescope exactly to the final spectrum in every cell, but in a very thick cell
 * whether a re-emitted packet is absorbed there again depends on where in the cell it is, and that
 * correlation depends on the order of the events. A run with many of its packets in flight at once
 * (one per GPU thread) is therefore not the one-packet-after-another run of the method: with 12 % of a
 * 1e6-packet run in flight, the inner-rim midplane of a tau_mid = 1e5 disk came out 17 % too hot and
 * escape-spectrum bins shifted by up to 20 %; with 0.03 % in flight the largest shift was 1.6 %, within
 * the noise of its reference. So with non-gray dust and max_in_flight = 0, at most
 * n_total / MCRT_NONGRAY_IN_FLIGHT packets are in flight (at least one warp); gray dust, whose
 * trajectories no temperature changes, uses the whole device. Batches interleave their models' packets
 * so that each model keeps this share. */
#define MCRT_NONGRAY_IN_FLIGHT 3000

typedef struct {
  int precision;                /* 32: production path; 64: debug path whose gray trajectories match
                                   the FP64 oracle event by event */
  int mrw;                      /* 1: modified random walk on (Sect. 2.2.2) */
  double gamma;                 /* Eq. 11: MRW only where d_min > gamma / (rho chi_R) */
  int mrw_min_interactions;     /* interactions in the current cell before the MRW may start (20) */
  int mrw_exit_dir;             /* direction after a jump: 0 isotropic, 1 cosine-weighted outward */
  uint64_t max_events_per_packet; /* a packet that exceeds this is dropped and counted as capped
                                     (values above 2^31 are taken as 2^31) */
  uint64_t n_total_packets;     /* packets of the whole run (energy per packet (L_star + internal
                                   sources) / n_total);
                                   0 means the n_packets of this call */
  int block_size;               /* threads per block of the transport kernel (multiple of 32, <= 256);
                                   0: tuned default */
  int refill_interval;          /* steps between refills of finished lanes; 0: the default (8 for a single
                                   disk, tuned for a batch) */
  int want_sed;                 /* gray dust only: 0 skips the emission-bin sampling (no SED) */
  int tail_warps_per_sm;        /* single-disk runs: the packets still in flight when the packet queue
                                   drains finish one per warp, this many warps per SM (0: 20; -1: no
                                   tail kernel, they finish in the transport kernel) */
  int interact_batch;           /* a warp runs the interaction code once this many of its lanes wait at
                                   an interaction point (or none can move on); 1: no waiting; 0: 8 */
  uint64_t max_in_flight;       /* at most this many packets in flight at once (the transport launch's
                                   threads, rounded up to whole blocks); 0: one per thread the device
                                   holds for gray dust, n_total / MCRT_NONGRAY_IN_FLIGHT for non-gray
                                   dust (see there) */
} mcrt_run_opts;

void mcrt_default_run_opts(mcrt_run_opts *o);

typedef struct {
  uint64_t packets, events, absorptions, scatterings, crossings, mrw_jumps, capped, escaped;
  uint64_t deposit_sum; /* sum over packets of their own fixed-point deposits: equals the growth of the
                           summed tallies when no update was lost */
  uint32_t error_flags; /* bit 0 deposit sum passed 2^64, bit 1 MRW deposit clipped, bit 2 step guard */
  double seconds;       /* device time of the transport kernel(s) */
  uint64_t max_packet_steps;  /* interactions + jumps + face crossings of the longest packet */
  uint64_t longest_packet;    /* its packet id modulo 2^24 */
  /* Step guards: a packet that takes more than 4 max_events_per_packet + 1e7 steps, or crosses 1e5
   * faces without an interaction, is dropped (counted in `capped` and `guarded`, error_flags bit 2).
   * The first one is recorded (single-disk runs) so that it can be replayed: */
  uint64_t guarded;           /* packets dropped by a step guard */
  uint64_t guard_packet;      /* full id of the first of them */
  int32_t guard_kind;         /* 0 none, 1 step limit, 2 face crossings without an interaction */
  int32_t guard_in_tail;      /* 1 if the tail kernel carried it */
  int32_t guard_cell[2];      /* its cell (ir, itheta) when the guard fired; ir = -1: inner cavity */
  uint64_t guard_events, guard_steps;  /* its interactions + jumps and its steps then */
  double guard_pos_cm[3];     /* its position (cm) and direction then */
  double guard_dir[3];
} mcrt_run_stats;

/* Transports packets first_packet_id .. first_packet_id+n_packets-1 (Sect. 2.1, 2.2.2): launch from
 * the star, optical-depth sampling, cell marching, scattering, absorption with immediate re-emission
 * into the 64-bit tallies, MRW jumps, escape into the spectrum tally. Packet k draws from the
 * Philox4x32-10 stream keyed by `seed`, counter (block, model 0, k). Tallies accumulate across calls
 * (resume from a checkpoint by continuing the packet ids). Synchronous; stats may be NULL. */
mcrt_status mcrt_run_photons(mcrt_disk *d, uint64_t n_packets, uint64_t seed, uint64_t first_packet_id,
                             const mcrt_run_opts *opts, mcrt_run_stats *stats);

/* Runs several disks in one persistent launch over a shared packet queue. Disk i transports
 * n_packets[i] packets from id 0 with Philox counter (block, model i, k). All disks must be on the
 * same device. stats: n entries or NULL. */
mcrt_status mcrt_run_batch(mcrt_disk *const *disks, int n, const uint64_t *n_packets, uint64_t seed,
                           const mcrt_run_opts *opts, mcrt_run_stats *stats);

/* A prepared batch: many disks (uneven grids and packet budgets) transported by one persistent launch
 * over a shared packet queue, captured once as a CUDA graph and replayed. Disk i draws from the Philox
 * counter (block, model i, k), k = 0 .. n_packets[i]-1, and its packet energy is L_star / n_packets[i].
 * When opts->block_size == 0 the batch is autotuned on creation: block size (64, 128, 256) and refill
 * interval (1, 4, 16) are timed on a short run (about 5 % of the packets) and the fastest is kept;
 * the tuning runs are then removed again by zeroing the disks' tallies. All disks must share one device;
 * the batch runs on the first disk's stream and must be destroyed before the disks. */
typedef struct mcrt_batch mcrt_batch;
mcrt_status mcrt_batch_create(mcrt_disk *const *disks, int n, const uint64_t *n_packets, const mcrt_run_opts *opts,
                              mcrt_batch **out);
/* Replays the graph with `seed` (synchronous); tallies accumulate like mcrt_run_photons. stats: n entries
 * or NULL. */
mcrt_status mcrt_batch_run(mcrt_batch *b, uint64_t seed, mcrt_run_stats *stats);
/* The launch configuration chosen (block size, refill interval, grid) and the tuning time (s). */
mcrt_status mcrt_batch_config(const mcrt_batch *b, int *block_size, int *refill_interval, int *grid,
                              double *tune_seconds);
void mcrt_batch_destroy(mcrt_batch *b);

/* Zeroes the tallies, visit counts and spectrum. */
mcrt_status mcrt_reset(mcrt_disk *d);

enum { MCRT_T_MC = 0, MCRT_T_PDA = 1 };
/* Flag for mcrt_raytrace's `which`: add the scattered light of the mean-intensity tally. */
enum { MCRT_WITH_SCATTERING = 4 };

/* Radiative-equilibrium temperature per cell (Sect. 2.1): solves 4 pi m kappa_P(T) B(T) = L_abs with
 * L_abs = tally / EUNIT * L_star / n_total. which = MCRT_T_MC: Monte Carlo temperatures; MCRT_T_PDA:
 * after mcrt_solve_pda, with the diffusion solution in the PDA cells. rel_err: statistical error
 * 1/(4 sqrt(N)), N = tally / EUNIT absorbed packet energies (infinity where N = 0). visits: packet
 * entries per cell. Host buffers of nr*ntheta; rel_err and visits may be NULL. */
mcrt_status mcrt_temperatures(mcrt_disk *d, int which, double *T_K, double *rel_err, uint64_t *visits);
mcrt_status mcrt_temperatures_dev(mcrt_disk *d, int which, double *T_K_dev, double *rel_err_dev);

/* Raw integer tallies (host buffers of nr*ntheta; each may be NULL). */
mcrt_status mcrt_get_tallies(mcrt_disk *d, uint64_t *tally, uint64_t *visits, uint64_t *n_absorptions);

/* Escaped luminosity per wavelength bin and inclination bin, L[lam * n_incl + i] (erg/s carried by
 * the packets that left r_out in that bin; multiply by n_incl for the isotropic equivalent).
 * n_incl must divide MCRT_NINC. */
mcrt_status mcrt_sed(mcrt_disk *d, int n_incl, double *L);

typedef struct {
  int min_visits;          /* PDA where fewer packets entered the cell (30, Sect. 3.1) */
  double max_rel_err;      /* ... or where the statistical T error exceeds this (0.05) */
  double tol;              /* relative FP64 residual of the refined solution (1e-12) */
  double inner_tol;        /* relative residual reduction of each FP32 inner solve (1e-5) */
  int max_outer;           /* FP64 refinement steps (50) */
  int max_inner;           /* FP32 CG iterations per refinement step (20000) */
  double min_cell_tau;     /* only cells at least this optically thick take part: rho * max_b chi'_b *
                              min(dr, r dtheta) >= min_cell_tau (1.0); diffusion needs optical depth */
  const double *kappa_R;   /* optional host array nr*ntheta: Rosseland extinction (cm^2/g) entering
                              D = 1/(3 rho kappa_R); NULL: from the dust at the MC temperature */
  const double *rho;       /* optional host array nr*ntheta: density (g/cm^3) entering D only; the PDA
                              region and the Monte Carlo boundary values stay those of the disk.
                              NULL: the disk's density. Used to differentiate with respect to rho. */
} mcrt_pda_opts;

void mcrt_default_pda_opts(mcrt_pda_opts *o);

/* Partial diffusion approximation (Sect. 2.2.1, Eq. 4 with D of Eq. 2): selects the PDA cells from
 * the visit counts and errors (among the optically thick cells), assembles face conductances (series resistance of half cells), and
 * solves for T^4 with an FP32 Jacobi-preconditioned conjugate gradient under FP64 iterative
 * refinement. Zero flux through grid edges and into dust-free cells. Afterwards MCRT_T_PDA
 * temperatures are available. out_n_pda_cells, out_iters (total inner iterations) may be NULL.
 * MCRT_EINVAL if a connected PDA region touches no Monte Carlo cell. */
mcrt_status mcrt_solve_pda(mcrt_disk *d, const mcrt_pda_opts *opts, int *out_n_pda_cells, int *out_iters);

/* Adjoint of the last PDA solve. For J = sum_i w_i T_i (T after the PDA, Monte Carlo boundary values
 * held fixed) returns dJ/dlog(rho_i) and dJ/dkappa_R,i per cell, through one more solve with the
 * (symmetric) PDA matrix. Host arrays of nr*ntheta; outputs may be NULL. */
mcrt_status mcrt_pda_adjoint(mcrt_disk *d, const double *w, double *grad_log_rho, double *grad_kappa_R);
mcrt_status mcrt_pda_adjoint_dev(mcrt_disk *d, const double *w_dev, double *grad_log_rho_dev,
                                 double *grad_kappa_R_dev);

/* Vertical hydrostatic structure (Sect. 2.5, Eq. 20): dP/dz = -rho G M_star z / R^3 with P = k_B rho T /
 * (mu m_u), at fixed surface density, from the disk's last temperatures. Each radial shell is one
 * column (z = r_c cos theta_c, R = r_c sin theta_c at the cell centres; trapezoid rule in z from
 * theta = 0 to pi) and keeps its dust mass; cells without dust stay without dust. One GPU thread per
 * shell, FP64. The paper iterates transport -> temperatures -> this density until the mean change of
 * the temperatures between two iterations is below 3 sigma of their Monte Carlo errors. */
typedef struct {
  double M_star_g;              /* stellar mass (g); default 2.5 solar masses (the paper's Table 1) */
  double mu;                    /* mean molecular weight (2.3) */
  double T_floor_K;             /* temperatures below this (cells no packet heated) are raised to it (10 K) */
  int which;                    /* MCRT_T_PDA (the last PDA solve, default) or MCRT_T_MC */
  const double *shell_mass_g;   /* optional host array nr: the dust mass each radial shell keeps;
                                   NULL: the disk's current shell masses */
  const double *relax;          /* optional host array nr, each in (0, 2]: a damped step per shell,
                                   log rho_new = (1 - a) log rho_cur + a log rho_Eq20 in the dusty cells,
                                   rescaled to the shell's mass (the paper iterates undamped); NULL: a = 1 */
} mcrt_hydro_opts;

void mcrt_default_hydro_opts(mcrt_hydro_opts *o);

/* New density (g/cm^3, host array nr*ntheta, row-major [ir][itheta]) in hydrostatic equilibrium with
 * the disk's temperatures. The disk is not changed (see mcrt_set_density). MCRT_ESTATE without
 * temperatures (or without a PDA solution for MCRT_T_PDA); MCRT_EINVAL for bad options. */
mcrt_status mcrt_hydrostatic_density(mcrt_disk *d, const mcrt_hydro_opts *opts, double *rho_out);

/* Replaces the disk's density (host array nr*ntheta, g/cm^3, finite and >= 0) and resets its tallies;
 * the grid, star and opacities stay. Device buffers keep their addresses. */
mcrt_status mcrt_set_density(mcrt_disk *d, const double *rho);

/* Internal sources (Sect. 5: viscous heating, whose energy the MRW carries out of the midplane):
 * luminosity per cell (host array nr*ntheta, erg/s, finite, >= 0, zero in dust-free cells; NULL or
 * all zero: none). Packets then start from the star or a cell in proportion to the luminosities and
 * carry (L_star + sum L) / N each; a cell's packet starts at a point uniform in the cell's volume and
 * is released there by an absorption with omega = 0, so its energy enters the cell's tally (the
 * temperatures then balance emission against absorption plus heating) and leaves with the
 * Bjorkman-Wood spectrum. Random draws: one extra block before each packet's launch (see
 * mcrt_run_photons). Resets the tallies; checkpoints do not hold the sources. MCRT_EINVAL for bad
 * values. */
mcrt_status mcrt_set_sources(mcrt_disk *d, const double *L_cell_erg_s);

/* Polarized transport (Sect. 2.3: the full angle-dependent Mueller matrix of each scattering). table:
 * host array [nlam][4][nmu] of S11, S12, S33, S34 at the scattering angles theta_k = k pi / (nmu - 1)
 * (S22 = S11, S44 = S33), linear in theta between them; finite, S11 >= 0 and not all zero; nmu in
 * 2 .. 4097; NULL turns polarization off. Packets then carry Stokes (Q, U, V) / I relative to a reference
 * vector: a scattering draws its angle from S11 sin(theta) and the azimuth of its plane from
 * 1 + (S12/S11)(q cos 2phi + u sin 2phi) with the two direction uniforms of its random block, and
 * applies the matrix; re-emitted packets and packets leaving an MRW sphere are unpolarized; escaping
 * packets add Q/I and U/I, in the frame of the disk axis projected on the sky, to fixed-point tallies
 * (2^20 per packet; read with mcrt_sed_stokes). Single disks only (batches and event traces refuse
 * polarized disks, MCRT_EINVAL); resets the tallies; checkpoints hold neither the matrix nor the Stokes
 * tallies. */
mcrt_status mcrt_set_mueller(mcrt_disk *d, int nmu, const double *table);

/* Escaped luminosity per (wavelength bin, inclination group) as Stokes I, Q, U (erg/s, each
 * nlam * n_incl host values, n_incl dividing MCRT_NINC), Q > 0 for light polarized along the projected
 * disk axis. MCRT_ESTATE without a Mueller matrix. */
mcrt_status mcrt_sed_stokes(mcrt_disk *d, int n_incl, double *L_I, double *L_Q, double *L_U);

/* ---- Ray-traced observables (Sect. 2.3: the observables come from integrating the computed source
 * function along rays, free of Monte Carlo noise; Sect. 4.1: SED from 0.1 um to 1 cm at 45 degrees,
 * N-band visibilities at a 100 m baseline). Readings: the source function of a cell in bin b is
 * kappa_b Bbar_b(T) / (kappa_b + sigma_b) with the cell's Monte Carlo temperature (the PDA temperatures
 * on request); scattering dims a ray, and adds the scattered light with MCRT_WITH_SCATTERING (below);
 * the star is a point source at the origin, dimmed along the radial line towards the observer, and
 * occults no ray.
 * Observer: direction o = (sin i, 0, cos i) for inclination i from the disk axis; sky-plane axes
 * e1 = (0, 1, 0) (the projected major axis) and e2 = (-cos i, 0, sin i); a ray through sky point (p, q)
 * is X(s) = p e1 + q e2 + s o. At most 256 wavelength bins. */

/* Sets the rays of the observables: n sky points (p_cm, q_cm) and the sky-plane area w_cm2 (>= 0) each
 * stands for, host arrays copied to the device and kept until the next call; incl in [0, pi],
 * dist_cm > 0. MCRT_EINVAL for bad sizes or values (n in 1 .. 2^27), MCRT_ESTATE before
 * mcrt_set_opacity. */
mcrt_status mcrt_set_rays(mcrt_disk *d, double incl_rad, double dist_cm, int64_t n, const double *p_cm,
                          const double *q_cm, const double *w_cm2);

/* Mean intensity from the path lengths of the packets (Sect. 2.3: the scattering field of the observables;
 * the path-length estimator, Lucy 1999). keep = 1: the following runs add the length of every flight to
 * a tally per cell and wavelength bin (the bin the packet has in flight), and the path length c t of every
 * MRW walk (Eq. 9, c t = x R0^2 / D) spread over the bins with the weights of Eq. 10, eta_b / chi'_b
 * (dBbar_b/dT normalised, the fixed point of Eq. 13) at the cell's temperature when the walk starts,
 * so that 4 pi m sum_b kappa_b J_b gives back the absorption. keep = 0: no tally (the production
 * kernels). Single disks without polarization or event trace (those refuse it, MCRT_EINVAL); gray dust
 * with want_sed = 0 keeps every flight in its launch bin. Resets the tallies; checkpoints do not hold it.
 * Device memory: nr * ntheta * nlam doubles. MCRT_ESTATE before mcrt_set_opacity. */
mcrt_status mcrt_keep_mean_intensity(mcrt_disk *d, int keep);

/* J_out: host array nr * ntheta * nlam (cell-major, bins fastest), the mean intensity integrated over
 * each bin, J = E_pkt (sum of path lengths) / (4 pi V) in erg s^-1 cm^-2 sr^-1, E_pkt the packet
 * energy of the runs (zero before any run). MCRT_ESTATE without mcrt_keep_mean_intensity. */
mcrt_status mcrt_mean_intensity(mcrt_disk *d, double *J_out);

/* Traces the rays through the disk with the temperatures `which` (MCRT_T_MC, computed first if
 * needed, or MCRT_T_PDA after a PDA solve) in FP32 (precision 0 or 32) or FP64 (64). With
 * MCRT_WITH_SCATTERING or'ed into `which`, the source function adds the scattered light
 * (sigma_b / chi_b) J_b of the mean-intensity tally (isotropic scattering; MCRT_ESTATE without
 * mcrt_keep_mean_intensity). Outputs, each
 * optional (NULL): F_out[nlam] the flux per wavelength bin at the observer, sum_k w_k I_kb / d^2 plus
 * the star (erg s^-1 cm^-2, integrated over the bin); F_star_out[nlam] the star's part;
 * I_out[n * nlam] the intensity of every ray per bin (erg s^-1 cm^-2 sr^-1, ray-major);
 * n_segments the number of ray segments through dusty cells. The image stays on the device for
 * mcrt_visibilities. MCRT_ESTATE without rays (or PDA temperatures), MCRT_ETIMEOUT if a ray crossed
 * more than 4 (nr + ntheta) + 64 faces. Synchronous. */
mcrt_status mcrt_raytrace(mcrt_disk *d, int which, int precision, double *F_out, double *F_star_out,
                          double *I_out, uint64_t *n_segments);

/* Visibility amplitudes of the last traced image: for each j, bin bins[j], baseline baseline_cm[j] >= 0
 * at position angle pa_rad[j] (from e1 towards e2), spatial frequency B (cos PA, sin PA) / lambda_b with
 * lambda_b = sqrt(lambda_lo lambda_hi) of the bin; |V| = |sum_k w_k I_k exp(-2 pi i (u p_k + v q_k) / d)
 * / d^2 + F*| / (sum_k w_k I_k / d^2 + F*), F* the dimmed star when with_star is nonzero, else 0.
 * vis_out: n_vis host values. MCRT_ESTATE before mcrt_raytrace. */
mcrt_status mcrt_visibilities(mcrt_disk *d, int n_vis, const int *bins, const double *baseline_cm,
                              const double *pa_rad, int with_star, double *vis_out);

/* FP64 debug transport that records every event of the first n_packets packets: type (0 launch,
 * 1 cell entry, 2 scatter, 3 absorption, 4 MRW jump, 5 escape, 6 capped), cell (-1 outside the grid),
 * wavelength bin and position (cm, [packet][event][3]). Buffers hold n_packets * max_events entries;
 * n_events[k] is the number recorded for packet k. Tallies accumulate as in mcrt_run_photons. */
mcrt_status mcrt_trace_packets(mcrt_disk *d, uint64_t n_packets, uint64_t seed, uint64_t first_packet_id,
                               const mcrt_run_opts *opts, int max_events, int32_t *type, int32_t *cell,
                               int32_t *lam, double *pos, int32_t *n_events);

/* Checkpoint of the integer state (tallies, visits, absorptions, spectrum, packets done). buf == NULL:
 * *len receives the size needed. Restoring and continuing the packet ids reproduces a single run.
 * Layout, all uint64 in host byte order: a header of 8 words {0x4D43525443484B31, version 1, nr, ntheta,
 * nlam, packets done, bits of the double packet count that normalises the tallies, 0}, then per cell
 * (r-major) the tallies, the entry counts and the absorption counts, then the escaping-energy spectrum
 * (nlam x 10 inclination bins). mcrt_restore checks the header against the disk (MCRT_EINVAL) and
 * zeroes the tallies a checkpoint does not hold (polarization Stokes, mean-intensity path lengths). */
mcrt_status mcrt_checkpoint(mcrt_disk *d, void *buf, size_t *len);
mcrt_status mcrt_restore(mcrt_disk *d, const void *buf, size_t len);

/* The device's Philox4x32-10 uniforms u_0..u_{n-1} of packet `packet` (model 0), as the transport
 * kernel draws them; and the device MRW inverse escape-time table x(P0) (Eq. 7-8). Test hooks. */
mcrt_status mcrt_debug_uniforms(int device, uint64_t seed, uint32_t model, uint64_t packet, int n, double *out);
mcrt_status mcrt_debug_mrw_x(int device, int n, const double *P0, double *x_out);

/* PDA solve that allocates nothing (the paper has no counterpart: this is a deployment variant of
 * mcrt_solve_pda's solver). Some callers may not allocate device memory once they are running -- a host
 * framework that owns every device byte through its own pool, or a service that fixes its memory at
 * start-up -- and mcrt_solve_pda allocates its working vectors on first use. This entry point takes the
 * assembled system in the caller's device buffers and keeps its working vectors in one file-scope
 * device array of fixed size; it never calls cudaMalloc or cudaFree.
 *   device:     CUDA device whose copy of the array is used (current during the call; the caller's
 *               current device is restored before it returns).
 *   nr, ntheta: grid; nr * ntheta <= 131072, or MCRT_EINVAL.
 *   mask_dev:   int8 per cell: 2 unknown (PDA) cell, 1 cell with a fixed value, 0 no flux.
 *   Cr_dev:     conductance of the face between (ir, it) and (ir+1, it), per cell (last row unused).
 *   Ct_dev:     conductance of the face between (ir, it) and (ir, it+1), per cell (last column unused).
 *   u_dev:      T^4 per cell: fixed values on mask-1 cells (read), the solution on mask-2 cells
 *               (written; their input values are the starting guess, normally 0).
 *   opts:       tol, inner_tol, max_outer, max_inner (<= 20000); the other fields are not used. tol is
 *               relative to |S b|, the scaled right-hand side (the residual with the unknowns at 0), as
 *               in mcrt_solve_pda, whatever the starting guess.
 *   cuda_stream: stream to run on (NULL: the legacy default stream). The call returns when the solve
 *               has finished on that stream.
 * The first call on a device looks up the device address of the array (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture on the device. Every call shares the
 * one array and starts by clearing what must be zero, so calls that overlap on the GPU (two streams,
 * two threads) race and must not be issued. Errors: MCRT_EINVAL for sizes beyond the limit, NULL
 * pointers or a PDA cell without a conducting face; MCRT_ENOTCONV as mcrt_solve_pda. */
mcrt_status mcrt_pda_solve_static(int device, int nr, int ntheta, const signed char *mask_dev,
                                  const double *Cr_dev, const double *Ct_dev, double *u_dev,
                                  const mcrt_pda_opts *opts, void *cuda_stream, int *out_iters);

/* Number of kernels this disk has launched since it was created (transport, temperature, PDA). */
mcrt_status mcrt_launch_count(const mcrt_disk *d, uint64_t *n);

/* Sizes and sanity of a disk. */
mcrt_status mcrt_disk_info(const mcrt_disk *d, int *nr, int *ntheta, int *nlam);

/* Message of the last failure on this disk (d == NULL: of the last failure in this thread). */
const char *mcrt_last_error(const mcrt_disk *d);

void mcrt_disk_destroy(mcrt_disk *d);

#ifdef __cplusplus
}
#endif
#endif /* MCRT_H */
