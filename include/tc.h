/*
 * tc.h -- C ABI of libtc: Coulomb charges in the unit disk on one B300 GPU.
 *
 * The library computes, with hand-written CUDA kernels for sm_103a, the hot
 * path of the adaptive subdomain method for the Thomson problem in a disk
 * (Lavrov & Nikonov, "Lowest-known energy configuration of N = 100 000
 * Coulomb charges in a disk"):
 *   - the direct-sum energy of Eq. (hamiltonian), E = sum_{i<j} 1/|r_i - r_j|,
 *     with the hard wall of Eq. (potential) (V = 0 for |r| <= R = 1),
 *   - its analytic gradient and the local energies e_i of Sec. II C step 1,
 *   - the subdomain objective E_sub of Sec. II D and the projected local
 *     relaxation of many active sets against all N charges (Sec. II C step 4,
 *     Sec. II E: n_act rows against the full configuration).
 *
 * Conventions for every call:
 *   - Positions are interleaved (x, y) float64 pairs: pos[2i], pos[2i+1].
 *   - Every array pointer is a DEVICE pointer owned by the caller, 16-byte
 *     aligned for position/gradient arrays, 8-byte aligned otherwise.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *     default stream).  Argument errors are returned synchronously; errors
 *     found on the device (coincident charges, non-finite values, charges
 *     outside the disk, invalid index sets) are recorded in a per-device
 *     status word that tc_sync_status() returns and clears.
 *   - The library keeps one scratch workspace per (device, stream), grown on
 *     demand with cudaMalloc and released by tc_shutdown().  The first call on
 *     a stream with a given size allocates; later calls of that size or
 *     smaller do not.
 *   - Gradients are dE/dr (the force is -grad).
 *   - n <= 1 gives E = 0 and zero gradients.
 *   - Charges closer than about 1e-19 are reported as coincident.
 */
#ifndef TC_H
#define TC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same object type as cudaStream_t, without requiring the CUDA headers. */
typedef struct CUstream_st* tc_stream;

typedef enum {
    TC_OK = 0,
    TC_ERR_INVALID_ARG = 1,   /* bad size, null or misaligned pointer, bad index set */
    TC_ERR_CUDA = 2,          /* a CUDA runtime call failed */
    TC_ERR_NONFINITE = 3,     /* coincident charges or NaN/Inf in the result */
    TC_ERR_OUTSIDE_DISK = 4,  /* a charge with |r| > 1 + 1e-12 (Eq. potential) */
    TC_ERR_TIMEOUT = 5,       /* a bounded device wait expired */
    TC_ERR_NOT_CONVERGED = 6, /* reserved: relaxation did not reach its tolerance */
    TC_ERR_NO_MEMORY = 7      /* workspace allocation failed */
} tc_status;

typedef enum {
    TC_FP64 = 0,  /* every pair term and sum in float64 */
    TC_MIXED = 1, /* pair terms in float32 from hi/lo-split positions, tile sums
                     in float32, cross-tile sums double-float, rows combined in float64 */
    TC_F64X = 2   /* float64-grade results from float32 arithmetic: positions split in
                     three float32 parts (exact separations), pair terms and tile sums in
                     double-float (~2^-46 relative per term), rows combined in float64;
                     held to the float64 tolerances (1e-13 energy, 1e-12 gradient) */
} tc_precision;

/* Launch shapes of the pair passes (tuning; the paper has no counterpart).
 * Every shape computes the same sums in the same order: a row block of 512
 * charges against tiles of 256 sources, the units (row block x tile) cut into
 * ranges whose number depends on the work and the SM count only (the mixed
 * passes take the ranges from a queue); shapes differ in CTA size, rows per
 * thread and CTAs per SM.  tc_pass_config_count(prec) shapes exist (0 .. count-1);
 * tc_set_pass_config selects one for every later call in this process
 * (TC_ERR_INVALID_ARG for an unknown shape); the default is 0.  An autotuner
 * (paper_2609_24722_b300/autotune.py) times the shapes and picks one. */
int32_t tc_pass_config_count(tc_precision prec);
tc_status tc_set_pass_config(tc_precision prec, int32_t config);
int32_t tc_get_pass_config(tc_precision prec);

/* Human-readable name of a status code (static storage). */
const char* tc_status_string(tc_status s);

/* Text of the last CUDA runtime failure that a call from this host thread
 * reported as TC_ERR_CUDA: the failing step and CUDA's error name/string
 * ("" if none).  Static thread-local storage, valid until the next call. */
const char* tc_last_error(void);

/* Waits for `stream`, then returns and clears the current device's status word. */
tc_status tc_sync_status(tc_stream stream);

/* Frees every workspace of every device this process used, and the kept
 * executable step-loop graphs. */
void tc_shutdown(void);

/* Total energy, Eq. (hamiltonian):  E = sum_{i<j} 1/|r_i - r_j|.
 *   pos      [2n]  positions (read)
 *   n              number of charges, n >= 0
 *   prec           TC_FP64, TC_F64X or TC_MIXED
 *   energy   [1]   E (written)
 *   local_e  [n]   nullable; e_i = 1/2 sum_{j != i} 1/|r_i - r_j|
 *                  (Sec. II C step 1), so sum_i e_i = E
 * Device errors: TC_ERR_NONFINITE, TC_ERR_OUTSIDE_DISK. */
tc_status tc_energy(const double* pos, int64_t n, tc_precision prec, double* energy,
                    double* local_e, tc_stream stream);

/* Gradient of Eq. (hamiltonian):  grad_i = dE/dr_i = sum_{j != i} -(r_i - r_j)/|r_i - r_j|^3.
 *   pos    [2n]  positions (read)
 *   grad   [2n]  dE/dr (written, interleaved like pos)
 *   energy [1]   nullable; E computed in the same pass
 * Device errors: TC_ERR_NONFINITE, TC_ERR_OUTSIDE_DISK. */
tc_status tc_grad(const double* pos, int64_t n, tc_precision prec, double* grad, double* energy,
                  tc_stream stream);

/* Energy change of moving each subdomain's active set, summed directly as pair
 * differences in float64 (never as a difference of totals).  For subdomain s
 * with active set A = idx[offsets[s] .. offsets[s+1]) and new positions
 * a_k = new_active[2 offsets[s] + 2k ..]:
 *   delta[s] = sum_{i in A, j not in A} (1/|a_i - p_j| - 1/|p_i - p_j|)
 *            + sum_{i<k in A} (1/|a_i - a_k| - 1/|p_i - p_k|)
 *            = E_sub(new) - E_sub(old)   (Sec. II D)
 * Each subdomain is evaluated against `pos` independently.
 *   pos        [2n]             configuration p (read)
 *   idx        [offsets[n_sub]] active indices, strictly ascending within a subdomain
 *   offsets    [n_sub + 1]      int64 CSR offsets, offsets[0] = 0, non-decreasing
 *   new_active [2 offsets[n_sub]] new positions of the active charges
 *   delta      [n_sub]          written
 * Device errors: TC_ERR_INVALID_ARG (index set), TC_ERR_NONFINITE. */
tc_status tc_subdomain_delta_energy(const double* pos, int64_t n, const int32_t* idx,
                                    const int64_t* offsets, int32_t n_sub, const double* new_active,
                                    double* delta, tc_stream stream);

/* The same energy change in the difference form, evaluated in float32 (the
 * paper has no counterpart: it is the float32 variant of E_sub(new) -
 * E_sub(old) of Sec. II D that stays accurate for small moves).  For a pair
 * with old separation d whose separation moves by u (d' = d + u),
 *     1/|d'| - 1/|d| = -u.(d + d') / (|d| |d'| (|d| + |d'|)),
 * so the result carries an error proportional to the moves, not to E_sub:
 *     |delta[s] - exact| <= bound[s] = 2^-15 sum over the pairs of |u|_a (1/|d| + 1/|d'|) / |d'|,
 * |u|_a the L1 norm of the moves entering u (valid for separations above ~1e-6;
 * a pair that ends nearly on top of another charge makes the bound huge).
 * Float64 pair differences (tc_subdomain_delta_energy) instead lose about
 * 1e-16 E_sub to cancellation, which dominates when the moves are small.
 *   arguments as tc_subdomain_delta_energy; bound [n_sub] device, nullable.
 * A pair whose float32 separation is exactly zero gives TC_ERR_NONFINITE. */
tc_status tc_subdomain_delta_energy_mixed(const double* pos, int64_t n, const int32_t* idx,
                                          const int64_t* offsets, int32_t n_sub, const double* new_active,
                                          double* delta, double* bound, tc_stream stream);

/* Gradient of the subdomain objective E_sub of Sec. II D, and its local
 * energies, for many subdomains at once: the pair pass that every step of
 * tc_relax_subdomains runs, evaluated once.  For subdomain s with active set
 * A = idx[offsets[s] .. offsets[s+1]) whose charges sit at
 * a_k = act[2 offsets[s] + 2k ..] (act NULL: a_k = pos[idx[k]]) while every
 * other charge j (the fixed set F) sits at pos[j]:
 *   grad[k]  = dE_sub/da_k = sum_{j in F} -(a_k - p_j)/|a_k - p_j|^3
 *                          + sum_{l in A, l != k} -(a_k - a_l)/|a_k - a_l|^3
 *   local_e[k] = e_k = sum_{j in F} 1/|a_k - p_j| + 1/2 sum_{l in A, l != k} 1/|a_k - a_l|
 *   e_sub[s] = E_sub = sum_{k in A} e_k
 * Subdomains are evaluated independently against pos (they may overlap).
 *   pos      [2n]               configuration (read)
 *   idx      [offsets[n_sub]]   active indices, strictly ascending within a subdomain
 *   offsets  [n_sub + 1]        int64 CSR offsets, offsets[0] = 0, non-decreasing
 *   act      [2 offsets[n_sub]] nullable: positions of the active charges
 *   prec     TC_FP64, TC_F64X or TC_MIXED (the float32 pair terms of the relaxation's bulk steps)
 *   grad     [2 offsets[n_sub]] written, interleaved like pos
 *   local_e  [offsets[n_sub]]   nullable, written
 *   e_sub    [n_sub]            nullable, written
 * Device errors: TC_ERR_INVALID_ARG (index set), TC_ERR_NONFINITE, TC_ERR_OUTSIDE_DISK. */
tc_status tc_subdomain_grad(const double* pos, int64_t n, const int32_t* idx, const int64_t* offsets,
                            int32_t n_sub, const double* act, tc_precision prec, double* grad, double* local_e,
                            double* e_sub, tc_stream stream);

/* Hard wall of Eq. (potential) as a projection, in place:
 *   r <- r min(1, radius/|r|);  a charge with flags[i] != 0 is pinned to the
 *   unit circle (the boundary population of Sec. II B): r <- r/|r| (unchanged
 *   at the origin).
 *   pos   [2n] in/out;  radius > 0;  flags [n] nullable. */
tc_status tc_project_disk(double* pos, int64_t n, double radius, const uint8_t* flags, tc_stream stream);

typedef enum {
    TC_OPT_GD = 0,    /* projected gradient descent x <- P(x - step0 g) */
    TC_OPT_BB = 1,    /* projected descent with Barzilai-Borwein (s^T y / y^T y) steps */
    TC_OPT_LBFGS = 2, /* L-BFGS on the smooth wall map x = radius sin|z| z/|z| (no projection) */
    TC_OPT_LBFGS_TU = 3, /* L-BFGS on the paper's (t, u) (Sec. II D): x = radius sin^2 t (cos u, sin u),
                           pinned (cos u, sin u); gradients by the paper's chain rule */
    TC_OPT_LBFGSB_TU = 4 /* L-BFGS-B (Byrd, Lu, Nocedal & Zhu 1995), the optimiser Sec. II C step 4
                            names, on the same (t, u) with the box t in [0, pi/2]: generalized
                            Cauchy point, direct-primal subspace minimisation, then the capped
                            step (and line search) below.  memory 1..8; one CTA steps each
                            problem, so a problem of many thousand charges steps slowly;
                            rms is the RMS of the projected gradient P(v - g) - v */
} tc_optimizer;

typedef struct {
    int32_t precision;   /* tc_precision of the bulk steps (TC_MIXED, TC_FP64 or TC_F64X) */
    int32_t optimizer;   /* tc_optimizer */
    int32_t n_steps;     /* bulk steps per problem (>= 0) */
    int32_t memory;      /* L-BFGS history pairs, 1..16 */
    double step0;        /* GD step; BB first step; L-BFGS scale without history */
    double alpha_min;    /* BB step clamp */
    double alpha_max;
    double maxstep;      /* L-BFGS: largest move of one charge in z per step */
    double gtol;         /* a problem stops once its RMS stationarity < gtol (0: never) */
    double radius;       /* wall radius for free charges (1 = the unit disk) */
    int32_t polish_steps;/* float64 L-BFGS steps after the bulk phase (0: none) */
    int32_t accept;      /* subdomain mode: 1 = sequential float64 accept/reject;
                            instance mode: 1 = write back only if E drops */
    double polish_gtol;  /* stopping tolerance of the float64 polish */
    int32_t want_energy; /* 1: also report each problem's final float64 E_sub / E */
    int32_t profile;     /* 1: launch the step loop directly (no CUDA graph) and time each
                            launch with CUDA events (see tc_relax_last_profile) */
    int32_t polish_precision; /* TC_FP64 (0, the default) or TC_F64X for the polish steps */
    int32_t line_search; /* L-BFGS only: at most this many Armijo halvings per step, 0..30
                            (0: none).  A trial z + alpha d is kept once E(new) - E(old)
                            <= 1e-4 alpha (dE/dz . d), the energy change summed as pair
                            differences (float32 difference form in a TC_MIXED phase,
                            float64 otherwise); else alpha halves; the last trial is kept */
} tc_relax_params;

typedef struct {
    double delta_e;  /* float64 pairwise energy change of the relaxed move */
    double energy;   /* final float64 E_sub (subdomain) or E (instance), if requested */
    double rms;      /* final RMS stationarity measure */
    int32_t steps;   /* steps taken (bulk + polish) */
    int32_t status;  /* 0 rejected, 1 accepted/written, 2 skipped (overlap) */
} tc_subdomain_result;

/* Relax many problems in one batched call (Sec. II C step 4; Sec. II E).
 *
 * Subdomain mode (idx != NULL): problem s moves the charges
 * idx[offsets[s] .. offsets[s+1]) (strictly ascending, inside the world range)
 * while every other charge of its world range stays at its value on entry;
 * the objective is E_sub of Sec. II D.  Problems run concurrently and may
 * overlap.  With accept = 1 they are then visited in order: a problem sharing
 * a charge with an accepted one is skipped; otherwise its float64 pairwise
 * energy change against the current configuration is computed and the move
 * is applied iff it is negative.  With accept = 0 nothing is written to pos.
 *
 * Instance mode (idx == NULL): problem s is the independent configuration
 * pos[world[2s] .. world[2s+1]), all of whose charges move.
 *
 *   pos     [2n]        in/out configuration
 *   world   [2 n_sub]   int64 [begin, end) charge range per problem; nullable
 *                       in subdomain mode (= [0, n)), required in instance mode
 *   flags   [n]         nullable; nonzero = pinned to the unit circle
 *   prm                 HOST pointer to the parameters
 *   out     [n_sub]     DEVICE results
 * Synchronises `stream`: it reads the sizes to the host first and returns
 * when the results are written.  The step loop runs as a 64-step CUDA graph
 * replayed on `stream`; the executable graph is kept after the call, and a
 * later call whose step loop has the same shape updates it in place instead
 * of instantiating a new one.  With gtol (or polish_gtol) > 0, the host checks
 * between replays whether any problem still steps, and stops once none
 * does.  Called while `stream` is being captured, every step joins the
 * caller's graph instead.
 * Device errors: TC_ERR_INVALID_ARG (index set), TC_ERR_NONFINITE, TC_ERR_OUTSIDE_DISK. */
tc_status tc_relax_subdomains(double* pos, int64_t n, const int32_t* idx, const int64_t* offsets,
                              int32_t n_sub, const int64_t* world, const uint8_t* flags,
                              const tc_relax_params* prm, tc_subdomain_result* out, tc_stream stream);

/* ---- The adaptive optimisation cycle (Sec. II C) ----
 *
 * One cycle runs T subdomain optimisations.  Each picks a centre (step 3) --
 * with probability p_defect a defect charge found by the local-energy
 * threshold of step 2, otherwise a point drawn uniformly over the disk -- and
 * optimises the charges of a zone around it (step 4) against all the others.
 * The paper lets the zone radius r_zone oscillate periodically without giving
 * the law; here a zone is the m charges nearest to the centre, and m follows
 * a triangle wave between m_min and m_max.  Random numbers are inputs: three
 * uniforms in [0,1) per subdomain, so a cycle is reproducible bit for bit. */
typedef struct {
    double kappa;     /* defects: e_i > mu + kappa sigma_e (the paper's rule: kappa = -1) */
    double p_defect;  /* probability that a centre is a defect charge (the paper: 0.8) */
    double radius;    /* disk radius (> 0) */
    double wall_tol;  /* |r_i| >= radius - wall_tol marks a boundary charge: never a defect */
    int32_t m_min;    /* zone size at schedule position q = 0 mod period (>= 0) */
    int32_t m_max;    /* zone size at q = period / 2 mod period (>= m_min) */
    int32_t period;   /* schedule period in subdomains (>= 1) */
    int32_t phase;    /* schedule position of the first subdomain (>= 0) */
} tc_zone_params;

/* Zone sizes and CSR offsets of n_sub subdomains at schedule positions
 * phase .. phase + n_sub - 1: with q' = q mod period,
 *   m_q = min(n, m_min + floor(2 (m_max - m_min) min(q', period - q') / period)),
 * offsets[0] = 0, offsets[s+1] = offsets[s] + m_(phase+s).
 *   offsets [n_sub + 1]  HOST array, written.  Host-only; no GPU work. */
tc_status tc_zone_offsets(const tc_zone_params* prm, int64_t n, int32_t n_sub, int64_t* offsets);

/* Steps 2-3 of Sec. II C and the zone of step 4, for n_sub subdomains:
 *   mu, sigma_e = mean and population standard deviation of local_e over all n;
 *   defects D = { i : local_e[i] > mu + kappa sigma_e, |r_i| < radius - wall_tol and
 *     flags[i] == 0 }, in ascending i;
 *   subdomain s takes u = uniforms[3s .. 3s+2]:
 *     centre = r_(D[floor(u1 |D|)]) if u0 < p_defect and D is not empty, else
 *              sqrt(u1) radius (cos 2 pi u2, sin 2 pi u2);
 *     zone   = the m_s charges with the smallest (d^2, i), d^2 = (x_i - c_x)^2 +
 *              (y_i - c_y)^2 rounded as written (no fused multiply-add), listed
 *              in ascending i -- a valid idx range for tc_relax_subdomains.
 *   pos      [2n]          device positions
 *   local_e  [n]           device e_i (tc_energy's local_e)
 *   flags    [n]           device, nonzero = pinned boundary charge (never a defect); nullable
 *   uniforms [3 n_sub]     device, each in [0, 1)
 *   idx      [offsets[n_sub]] device, written (size it with tc_zone_offsets)
 *   offsets  [n_sub + 1]   device, written
 *   centres  [2 n_sub]     device, written; nullable
 *   stats    [3]           device, written (mu, sigma_e, |D|); nullable
 * Asynchronous on `stream`; TC_ERR_INVALID_ARG for bad sizes or parameters. */
tc_status tc_select_subdomains(const double* pos, int64_t n, const double* local_e, const uint8_t* flags,
                               const tc_zone_params* prm, int32_t n_sub, const double* uniforms, int32_t* idx,
                               int64_t* offsets, double* centres, double* stats, tc_stream stream);

typedef struct {
    tc_zone_params zone;    /* zone.phase: schedule position of the cycle's first subdomain;
                               zone.radius is replaced by the batch's sigma */
    tc_relax_params relax;  /* optimiser of step 4; accept is forced to 1, radius replaced by sigma */
    int32_t batch;          /* subdomains selected and relaxed together (1 = one at a time) */
    int32_t local_precision;/* tc_precision of the e_i that pick the centres */
    double sigma0;          /* interior radius of the first batch (Sec. II B); <= 0: Eq. sigma,
                               1 - 1/(2 sqrt(n)) ... */
    double sigma1;          /* ... rising linearly to this one at the last batch;
                               wall_tol < sigma0 <= sigma1 <= 1 (1, 1: the plain unit disk) */
    int32_t disjoint;       /* 0: a batch is the next `batch` subdomains; 1: it is the longest
                               prefix of pairwise disjoint zones among them (see tc_cycle) */
    int32_t ramp_first;     /* this call runs subdomains ramp_first .. ramp_first + n_sub - 1 of a */
    int32_t ramp_total;     /* cycle of ramp_total (0: of n_sub, ramp_first = 0): the sigma ramp runs
                               over the whole cycle, so a cycle run as several calls (a checkpoint
                               after each) takes the radii of one call; with fixed batches
                               ramp_first must be a multiple of `batch` */
} tc_cycle_params;

/* One optimisation cycle (Sec. II C) of n_sub subdomains, in batches of
 * `batch` consecutive ones.  For each batch: the local energies e_i of the
 * current configuration (step 1), tc_select_subdomains at schedule position
 * zone.phase + first subdomain of the batch (steps 2-3), then
 * tc_relax_subdomains with the sequential float64 accept (step 4).  batch = 1
 * recomputes e_i before every subdomain, as the paper's cycle does; a larger
 * batch relaxes its zones concurrently against the configuration at the
 * batch's start and accepts them in order.  Batch b of n_batches uses the
 * interior radius sigma_b = sigma0 + (sigma1 - sigma0) b / (n_batches - 1)
 * (sigma1 for one batch) for the free charges and for the zone centres and
 * boundary test; pinned charges (flags) move along the unit circle and are
 * never defects (Sec. II B).
 *   pos      [2n]          in/out configuration (device); free charges within sigma0
 *   flags    [n]           device, nonzero = pinned to the unit circle; nullable
 *   uniforms [3 n_sub]     device, each in [0, 1)
 *   out      [n_sub]       device results, as tc_relax_subdomains
 *   energy   [n_batches+1] device; E (in local_precision) before each batch and
 *                          after the last; nullable
 * With disjoint = 1 a batch is formed differently: the zones of the next
 * `batch` subdomains are selected, and the batch is their longest prefix of
 * pairwise disjoint zones (at least one zone).  The zones after that prefix
 * are dropped and selected again, from the configuration and local energies
 * after this batch, as the start of the next batch.  So no zone is skipped
 * by the accept, every drawn centre is optimised, and the relaxations of a
 * batch interact only through the long-range cross terms that the
 * sequential accept then evaluates exactly.  The interior radius of a batch
 * whose first subdomain is b0 is sigma0 + (sigma1 - sigma0) b0 / (n_sub - 1)
 * (sigma1 for n_sub = 1), and `energy` needs n_sub + 1 entries, of which the
 * first (batches run) + 1 are written.
 * Synchronises the stream once per batch (the zone sizes are host-known, the
 * relaxation reads its offsets back; the disjoint form reads its prefix
 * length).  Device errors as tc_relax_subdomains. */
tc_status tc_cycle(double* pos, int64_t n, const uint8_t* flags, const tc_cycle_params* prm, int32_t n_sub,
                   const double* uniforms, tc_subdomain_result* out, double* energy, tc_stream stream);

/* Eq. Nb (Sec. II B): the number of boundary charges,
 *   N_b = round(2.84328 N^(2/3) - 0.530196 N^(1/3) - 2.32866), within [0, n].
 * Host-only. */
int64_t tc_boundary_count(int64_t n);

/* The border-interior split of Sec. II B: ordering the charges by (|r|^2, i)
 * ascending, the last n_b become boundary charges pinned to the unit circle
 * (flags = 1, r <- r/|r|; unchanged at the origin) and the others interior
 * charges confined to radius sigma (flags = 0, r <- r min(1, sigma/|r|)).
 *   pos   [2n] device, in/out;  flags [n] device, written;
 *   0 <= n_b <= n;  sigma <= 1, where sigma <= 0 takes Eq. sigma, 1 - 1/(2 sqrt(n)).
 *   Asynchronous on `stream`. */
tc_status tc_border_split(double* pos, int64_t n, int64_t n_b, double sigma, uint8_t* flags, tc_stream stream);

/* Structure analysis of Sec. III C-D: Voronoi neighbours, the coordination
 * number z_i (the number of neighbours) and the sixfold bond-orientational
 * order of Eq. (psi6), psi6_i = (1/z_i) sum_{j in N(i)} exp(6 i theta_ij),
 * theta_ij the angle of the bond i -> j against the x axis.  Two charges are
 * Voronoi neighbours when their cells share an edge (equivalently, a Delaunay
 * edge joins them).  Each cell is built in float64 by clipping the square
 * [-1e6, 1e6]^2 with the bisectors of the charges that can still cut it, so
 * cells of charges on the convex hull are cut off at that square; a Voronoi
 * edge lying wholly outside it (three hull charges collinear to ~1e-6) would
 * be missed.
 *   pos     [2n]          device positions
 *   z       [n]           device int32, written
 *   psi6    [2n]          device (re, im) pairs, written; 0 for z_i = 0
 *   nbr     [n max_nbr]   device int32, nullable: neighbours of i ascending at
 *                         nbr[i max_nbr ..], -1 padded
 *   summary [18]          device, nullable: <|psi6|>, |<psi6>|, then P(z) for
 *                         z = 0 .. 15 (the last bin holds z >= 15)
 * Device errors: TC_ERR_NONFINITE (coincident charges), TC_ERR_INVALID_ARG
 * (a cell with more than 40 vertices while clipping, or z_i > max_nbr). */
tc_status tc_voronoi_order(const double* pos, int64_t n, int32_t* z, double* psi6, int32_t* nbr, int32_t max_nbr,
                           double* summary, tc_stream stream);

/* Total energy (and local energies) as tc_energy computes them for TC_FP64
 * and TC_MIXED (same pair kernels, same sums, within the same tolerances),
 * but without allocating any device memory.  The paper has no counterpart.
 * This entry point is for callers that cannot call cudaMalloc: processes
 * whose device memory is all handed out by a framework's own pool allocator,
 * and real-time or embedded hosts that forbid allocation after start-up
 * (cudaMalloc can block and synchronise the device).
 *   pos [2n], energy [1], local_e [n] (nullable): as for tc_energy.
 *   prec: TC_FP64 or TC_MIXED (TC_F64X returns TC_ERR_INVALID_ARG).
 *   n <= 200 000; larger n returns TC_ERR_INVALID_ARG (tc_last_error() says why).
 * Scratch: one fixed 16 MiB array in the library's device image, present on
 * every GPU that loads libtc until the process exits.  Every call shares it,
 * so calls that overlap on the GPU (other streams, other host threads) race:
 * the caller must order them.  Each call clears the part that must start at
 * zero.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current.  Device-side errors
 * (coincident charges, non-finite values, charges outside the disk, n = 1
 * included) make *energy NaN; they are not recorded in the status word that
 * tc_sync_status() reads. */
tc_status tc_energy_noalloc(const double* pos, int64_t n, tc_precision prec, double* energy,
                            double* local_e, tc_stream stream);

/* Launch timings of the calling thread's last tc_relax_subdomains call made
 * with prm->profile = 1 (measurement utility; the paper has no counterpart).
 * Times are CUDA-event intervals on the launching stream, in milliseconds. */
typedef struct {
    double pass_ms;     /* sum over the relaxation pair passes (bulk + polish) */
    double update_ms;   /* sum over the optimiser update launches */
    double relax_ms;    /* whole step loop(s) */
    double accept_ms;   /* energy-change passes and accept/apply launches */
    double setup_ms;    /* set-up launches before the first step */
    int32_t n_pass;     /* relaxation pair-pass launches */
    int32_t launches;   /* every kernel launch of the call */
    int64_t pass_pairs; /* ordered pair interactions of one bulk pass over all problems */
} tc_relax_profile;

tc_status tc_relax_last_profile(tc_relax_profile* out);

/* Measurement utility (the paper has no counterpart): achieved throughput of
 * the instruction pipes that bound the pair kernels, measured with long
 * chains of independent instructions on every SM of the current device.
 *   rates [4] HOST array, written: float32 FFMA lane operations/s,
 *             float64 DFMA operations/s, MUFU.RSQ operations/s, and ordered
 *             pairs/s of the far-tile pair instruction mix (packed float32
 *             differences, r^2, two MUFU.RSQ, r^-3, gradient fmas) run from
 *             registers with no memory traffic.
 * Synchronous; allocates and frees a 64-byte scratch buffer. */
tc_status tc_probe_pipes(double* rates, tc_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* TC_H */
