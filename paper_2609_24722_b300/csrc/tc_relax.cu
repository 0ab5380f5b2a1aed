// tc_relax.cu -- batched relaxation of subdomains / instances and the
// pairwise energy change of Sec. II D.
//
// A relaxation step of every problem is one pair pass (all problems' units in
// one persistent launch, tc_pass.cuh) followed by one update launch (one CTA
// per problem: reduce the row partials in a fixed order, take the optimiser
// step, re-split the moved rows; L-BFGS-B in tc_lbfgsb.cuh; L-BFGS of very
// large problems as grid-wide launches), and optionally an Armijo line search.
// 64 steps are captured once into a CUDA graph and replayed; with a stopping
// tolerance the host stops replaying once no problem is active.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <vector>

#include <cooperative_groups.h>

#include "tc_plan.cuh"

namespace tc {

namespace cg = cooperative_groups;

constexpr int kUpd = 256;   // update / reduction CTA size
constexpr int kMaxMem = 16; // largest L-BFGS memory
// Problems with more rows than this take the L-BFGS update (smooth map or
// (t, u)) as a sequence of grid-wide launches instead of one CTA; L-BFGS-B
// steps every problem on one CTA or one thread-block cluster (launch_lbfgsb).
constexpr int kLargeRows = 16384;
constexpr int kLargeBlocks = 296;  // CTAs of the grid-wide update launches
// Resident CTAs per SM of the queued one-CTA L-BFGS update (used when there
// are more problems than such CTAs).
constexpr int kUpdPerSm = 2;  // 2 beat 1 and 3 on C5 (512 instances): 0.47 s against 0.60 and 0.63 s a round
// Byte offset, in the workspace's counter area, of the update queue's ticket counter.
constexpr size_t kUpdCtrOff = 64;
// Gradient passes with more slots per row than this are summed by k_sum_slots
// (every SM) before the update kernels read them.
constexpr int64_t kPreReduceSlots = 16;
// Instances take their float64 passes symmetric (each unordered pair once,
// PassArgs::sym) when the source sums, 24 bytes per row and row block, fit this.
constexpr int64_t kSymBytes = int64_t(2) << 30;

struct RelaxDev {
    const Prob* prob;
    int S;
    int64_t M;
    const int64_t* wbeg;   // per problem: first charge of the world range
    const int32_t* idx;    // nullable (instance mode)
    const uint8_t* flags;  // nullable
    double2* pos;          // the caller's configuration
    int32_t* gidx;         // per row: charge index
    double2* x;            // per row: position (float64 master copy)
    float4* xs;            // per row: hi/lo split of x
    fx3* x3;               // per row: three-part split of x (float64-grade float32 pass), nullable
    double2* g;            // per row: reduced dE/dx
    double2* g_red;        // per row: the pass's slots summed (k_sum_slots), nullable
    double2* xp;           // per row: previous x (BB) / previous z (L-BFGS)
    double2* gp;           // per row: previous g (BB) / current dE/dz (L-BFGS)
    double2* z;            // per row: L-BFGS variable
    double2* q;            // per row: L-BFGS work vector
    double2* Sh;           // [mem][M] L-BFGS s history
    double2* Yh;           // [mem][M] L-BFGS y history
    d4* rows4;             // per row: (old, new) for the float64 energy change
    f8* rows8;             // per row: old split + move for the float32 difference form (line search)
    double2* xold;         // per row: x before the step (line search), nullable
    double* ls_alpha;      // per problem: current trial step scale (line search)
    double* ls_gd;         // per problem: dE/dz . d at the start of the step
    int* ls_active;        // per problem: 1 while its trial step is being tested
    uint32_t* mask;        // per problem: own-charge bit mask over its world range
    uint32_t* taken;       // over all n charges: charges moved by an accepted problem
    int* active;           // per problem: still stepping
    int* ok;               // per problem: take part in the energy-change pass
    int* steps;            // per problem
    int* hist;             // per problem: L-BFGS pairs stored
    int* head;             // per problem: L-BFGS ring position
    double* rho;           // [S][kMaxMem]: 1/(s_j.y_j) by ring slot
    double* gram;          // [S][2][kMaxMem][kMaxMem]: s_a.y_b and y_a.y_b by ring slot (L-BFGS)
    double* rms;           // per problem
    double* delta;         // per problem
    double* energy;        // per problem
    int* status;           // per problem
    int* st;               // device status word
    int tu;                // L-BFGS variables: 0 the smooth wall map, 1 the paper's (t, u)
    int boxed;             // 1: L-BFGS-B, every (t, u) point is kept inside the box t in [0, pi/2]
    double* bp;            // per row: breakpoint of the row's t in the Cauchy search (L-BFGS-B)
    double2* xc;           // per row: generalized Cauchy point (L-BFGS-B)
    double* bsmall;        // per problem: s.y and s.s of the stored pairs by slot, theta (L-BFGS-B)
    int* any_active;       // one int: some problem still steps (early stop between graph replays)
    const int32_t* upd_order;  // nullable: problems of the queued L-BFGS update, largest first
    int upd_n;                 // entries of upd_order
    int upd_ctas;              // CTAs of the queued update launch
    unsigned* upd_ctr;         // its ticket counter (zero between launches)
};

__device__ __forceinline__ int find_row_prob(const Prob* __restrict__ P, int S, int64_t row)
{
    int lo = 0, hi = S - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (P[mid].row_base <= row)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Row partial of one pass: sum of its slots in order (float64, compensated for e),
// then, after a symmetric float64 pass, the source sums that the earlier row
// blocks rb < t / 2 left for the row's tile t, in order of rb.
struct SlotView {
    int64_t W, G, u_base, stride, row_sub;
    const double2* red = nullptr;     // nullable: the rows' gradients already summed (k_sum_slots)
    const double2* colg = nullptr;    // nullable: source sums of a symmetric pass (PassArgs::col_g)
    const double* cole = nullptr;     // nullable: the same for 1/r (PassArgs::col_e)
    int64_t col_stride = 0;
    const double* rede = nullptr;     // nullable: the rows' energy partials already summed (k_sum_slots_e)
};

__device__ __forceinline__ double2 sum_g(const Prob& p, int64_t rl, const double2* part_g, const SlotView& v)
{
    if (v.red) return v.red[p.row_base + rl - v.row_sub];
    int64_t c = slot_count(p, (int)(rl / kRB), v.u_base, v.W, v.G);
    double gx = 0.0, gy = 0.0;
    int64_t o = p.row_base + rl - v.row_sub;
    for (int64_t k = 0; k < c; ++k) {
        double2 q = part_g[k * v.stride + o];
        gx += q.x;
        gy += q.y;
    }
    if (v.colg) {
        const int64_t nb = rl / kT / 2;
        for (int64_t b = 0; b < nb; ++b) {
            const double2 q = v.colg[b * v.col_stride + o];
            gx += q.x;
            gy += q.y;
        }
    }
    return make_double2(gx, gy);
}

__device__ __forceinline__ double sum_e(const Prob& p, int64_t rl, const double* part_e, const SlotView& v)
{
    if (v.rede) return v.rede[p.row_base + rl - v.row_sub];
    int64_t c = slot_count(p, (int)(rl / kRB), v.u_base, v.W, v.G);
    double hi = 0.0, lo = 0.0;
    int64_t o = p.row_base + rl - v.row_sub;
    for (int64_t k = 0; k < c; ++k) dd_add(hi, lo, part_e[k * v.stride + o]);
    if (v.cole) {
        const int64_t nb = rl / kT / 2;
        for (int64_t b = 0; b < nb; ++b) dd_add(hi, lo, v.cole[b * v.col_stride + o]);
    }
    return hi + lo;
}

// The reduction view of a gradient/energy pass launched with `a` over G ranges.
__host__ inline SlotView pass_view(const PassArgs& a, int64_t W, int64_t G, int64_t M)
{
    SlotView v{W, G, 0, M, 0};
    if (a.sym) {
        v.colg = a.col_g;
        v.cole = a.col_e;
        v.col_stride = a.col_stride;
    }
    return v;
}

// Deterministic block reductions of several doubles at once.
template <int N> __device__ void block_sums(double (&v)[N], double* sh)
{
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = block_sum<kUpd>(v[i], sh);
}

__device__ double block_max(double v, double* sh)
{
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = kUpd / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + w]);
        __syncthreads();
    }
    double r = sh[0];
    __syncthreads();
    return r;
}

// ------------------------------------------------------ wall parameterisation ---
// Free charge: x = radius sin|z| z/|z| (x = radius z as z -> 0).  Pinned charge:
// x = z/|z|.  The wall is a smooth maximum of |x|, as for the paper's
// r = sigma sin^2 t of Sec. II D, so L-BFGS needs no projection.

// Two L-BFGS variables for the wall.  The smooth map (tu = false): a free charge
// is z in R^2 with x = radius sin|z| z/|z|, a pinned one x = z/|z|.  The
// paper's parameterisation (tu = true, Sec. II D): a free charge is (t, u) with
// x = radius sin^2 t (cos u, sin u), a pinned one (u, 0) with x = (cos u, sin u).
// Both make the wall a smooth maximum of |x|, so neither needs a projection.
__device__ __forceinline__ double2 z_to_x(double2 z, double radius, bool pinned, bool tu)
{
    if (tu) {
        double s_, c_;
        if (pinned) {
            sincos(z.x, &s_, &c_);
            return make_double2(c_, s_);
        }
        const double st = sin(z.x), r = radius * st * st;
        sincos(z.y, &s_, &c_);
        return make_double2(r * c_, r * s_);
    }
    double rho = sqrt(z.x * z.x + z.y * z.y);
    if (pinned) return make_double2(z.x / rho, z.y / rho);
    if (rho > 0.0) {
        double f = radius * sin(rho) / rho;
        return make_double2(z.x * f, z.y * f);
    }
    return make_double2(0.0, 0.0);
}

__device__ __forceinline__ double2 x_to_z(double2 x, double radius, bool pinned, bool tu)
{
    double r = sqrt(x.x * x.x + x.y * x.y);
    if (tu) {
        const double u = r > 0.0 ? atan2(x.y, x.x) : 0.0;
        if (pinned) return make_double2(u, 0.0);
        return make_double2(asin(sqrt(fmin(r / radius, 1.0))), u);
    }
    if (pinned) return r > 0.0 ? make_double2(x.x / r, x.y / r) : make_double2(1.0, 0.0);
    if (r > 0.0) {
        double q = fmin(r / radius, 1.0);
        double f = asin(q) / r;
        return make_double2(x.x * f, x.y * f);
    }
    return make_double2(0.0, 0.0);
}

// dE/dz from dE/dx by the chain rule of the map above; for (t, u) these are
// the paper's dE/dt = (E_x cos u + E_y sin u) radius sin 2t,
// dE/du = -E_x r sin u + E_y r cos u (pinned: r = 1, and 0 for the unused second variable).
__device__ __forceinline__ double2 grad_z(double2 z, double2 g, double radius, bool pinned, bool tu)
{
    if (tu) {
        double sn, c;
        sincos(z.x, &sn, &c);
        if (pinned) return make_double2(-g.x * sn + g.y * c, 0.0);
        const double st = sn, ct = c;  // sin 2t = 2 sin t cos t
        sincos(z.y, &sn, &c);
        const double r = radius * st * st;
        return make_double2((g.x * c + g.y * sn) * radius * (2.0 * st * ct), (-g.x * sn + g.y * c) * r);
    }
    double rho = sqrt(z.x * z.x + z.y * z.y);
    if (rho == 0.0) return pinned ? make_double2(0.0, 0.0) : make_double2(radius * g.x, radius * g.y);
    // one reciprocal and one sincos: the float64 pipe is this update's limit
    const double ri = 1.0 / rho;
    double ux = z.x * ri, uy = z.y * ri;
    double gr = g.x * ux + g.y * uy;
    double tx = g.x - gr * ux, ty = g.y - gr * uy;
    if (pinned) return make_double2(tx * ri, ty * ri);
    double sn, c;
    sincos(rho, &sn, &c);
    const double a = sn * ri;
    return make_double2(radius * (a * tx + c * gr * ux), radius * (a * ty + c * gr * uy));
}

// ------------------------------------------------------------- set-up ---

__global__ void k_rows_init(RelaxDev d, int64_t n, double radius, int lbfgs)
{
    for (int64_t rr = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; rr < d.M; rr += (int64_t)gridDim.x * blockDim.x) {
        const int s = find_row_prob(d.prob, d.S, rr);
        const Prob p = d.prob[s];
        const int64_t rl = rr - p.row_base;
        int64_t j;
        bool bad = false;
        if (d.idx) {
            j = d.idx[rr];
            bad = j < p.snap_b || j >= p.snap_e || (rl > 0 && d.idx[rr - 1] >= j);
        } else {
            j = d.wbeg[s] + rl;
        }
        if (bad || j < 0 || j >= n) {
            set_status(d.st, ST_INVALID);
            j = 0;
        }
        d.gidx[rr] = (int32_t)j;
        double2 x = d.pos[j];
        if (!isfinite(x.x) || !isfinite(x.y)) set_status(d.st, ST_NONFINITE);
        else if (!inside(x.x, x.y)) set_status(d.st, ST_OUTSIDE);
        if (lbfgs) {
            const bool pinned = d.flags && d.flags[j];
            double2 z = x_to_z(x, radius, pinned, d.tu);
            if (d.boxed && !pinned) z.x = fmin(fmax(z.x, 0.0), 1.5707963267948966);
            x = z_to_x(z, radius, pinned, d.tu);
            d.z[rr] = z;
        }
        if (d.x) d.x[rr] = x;
        if (d.xs) d.xs[rr] = split4(x.x, x.y);
        if (d.x3) d.x3[rr] = split3(x.x, x.y);
    }
}

__global__ void k_mask_build(RelaxDev d)
{
    for (int64_t rr = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; rr < d.M; rr += (int64_t)gridDim.x * blockDim.x) {
        const int s = find_row_prob(d.prob, d.S, rr);
        const Prob p = d.prob[s];
        if (p.mask_off < 0) continue;
        int64_t j = (int64_t)d.gidx[rr] - p.snap_b;
        if (j < 0 || j >= p.snap_e - p.snap_b) continue;
        atomicOr(&d.mask[p.mask_off + (j >> 5)], 1u << (j & 31));
    }
}

__global__ void k_split_pos(const double2* __restrict__ pos, int64_t n, float4* __restrict__ out, int* st)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 p = pos[i];
        if (!isfinite(p.x) || !isfinite(p.y))
            set_status(st, ST_NONFINITE);
        else if (!inside(p.x, p.y))
            set_status(st, ST_OUTSIDE);
        out[i] = split4(p.x, p.y);
    }
}

__global__ void k_split3_pos(const double2* __restrict__ pos, int64_t n, fx3* __restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = split3(pos[i].x, pos[i].y);
}

// ------------------------------------------------------------ updates ---

struct StepParams {
    int opt;
    int memory;
    double step0, alpha_min, alpha_max, maxstep, gtol, radius;
    int measure;  // 1: only record the RMS stationarity of the current rows (no step)
    int line_search = 0;  // L-BFGS: at most this many Armijo halvings per step (0: none)
    int pre_reduce = 0;   // host: sum the pass's slots over all SMs first (k_sum_slots)
};

// Each row's gradient partials summed in slot order (sum_g) into d.g_red, over
// every SM, for passes with many slots per row: the update kernels, which run
// on few CTAs, then read one value per row.  The sums are those sum_g forms.
__global__ void k_sum_slots(RelaxDev d, const double2* __restrict__ part_g, SlotView v)
{
    for (int64_t rr = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; rr < d.M; rr += (int64_t)gridDim.x * blockDim.x) {
        const Prob p = d.prob[find_row_prob(d.prob, d.S, rr)];
        d.g_red[rr] = sum_g(p, rr - p.row_base, part_g, v);
    }
}

// The energy partials of problem s's rows summed in slot order (sum_e) into
// red[row - v.row_sub], one row per thread: the sequential accept's one-CTA
// kernel then reads one value per row.  Skipped when the problem is not active.
__global__ void k_sum_slots_e(RelaxDev d, int s, const double* __restrict__ part_e, SlotView v, double* red)
{
    if (!d.ok[s]) return;
    const Prob p = d.prob[s];
    const int64_t rl = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (rl < p.m) red[p.row_base + rl - v.row_sub] = sum_e(p, rl, part_e, v);
}

// Projected gradient descent (fixed or Barzilai-Borwein step), one CTA per problem.
__global__ void __launch_bounds__(kUpd) k_update_gdbb(RelaxDev d, const double2* __restrict__ part_g, SlotView v,
                                                       StepParams sp)
{
    __shared__ double sh[kUpd];
    const int s = blockIdx.x;
    if (!d.active[s]) return;
    const Prob p = d.prob[s];
    const int k = d.steps[s];
    double acc[3] = {0.0, 0.0, 0.0};  // |pg|^2, s.y, y.y
    bool bad = false;
    for (int64_t rl = threadIdx.x; rl < p.m; rl += kUpd) {
        const int64_t row = p.row_base + rl;
        double2 g = sum_g(p, rl, part_g, v);
        if (!isfinite(g.x) || !isfinite(g.y)) bad = true;
        d.g[row] = g;
        const double2 x = d.x[row];
        const bool pinned = d.flags && d.flags[d.gidx[row]];
        double2 pg = wall_grad(x, g, sp.radius, pinned);
        acc[0] += pg.x * pg.x + pg.y * pg.y;
        if (sp.opt == TC_OPT_BB && k > 0) {
            double2 xo = d.xp[row], go = d.gp[row];
            double sx = x.x - xo.x, sy = x.y - xo.y, yx = g.x - go.x, yy = g.y - go.y;
            acc[1] += sx * yx + sy * yy;
            acc[2] += yx * yx + yy * yy;
        }
    }
    if (bad) set_status(d.st, ST_NONFINITE);
    block_sums(acc, sh);
    const double rms = sqrt(acc[0] / (double)max(p.m, 1));
    if (sp.measure || (sp.gtol > 0.0 && rms < sp.gtol)) {
        if (threadIdx.x == 0) {
            if (!sp.measure) d.active[s] = 0;
            d.rms[s] = rms;
        }
        return;
    }
    double alpha = sp.step0;
    if (sp.opt == TC_OPT_BB && k > 0) {
        alpha = (acc[1] > 0.0 && acc[2] > 0.0) ? acc[1] / acc[2] : sp.alpha_max;
        alpha = fmin(fmax(alpha, sp.alpha_min), sp.alpha_max);
    }
    for (int64_t rl = threadIdx.x; rl < p.m; rl += kUpd) {
        const int64_t row = p.row_base + rl;
        const double2 x = d.x[row], g = d.g[row];
        const bool pinned = d.flags && d.flags[d.gidx[row]];
        d.xp[row] = x;
        d.gp[row] = g;
        double2 xn = make_double2(__dsub_rn(x.x, __dmul_rn(alpha, g.x)), __dsub_rn(x.y, __dmul_rn(alpha, g.y)));
        xn = project1(xn, sp.radius, pinned);
        d.x[row] = xn;
        d.xs[row] = split4(xn.x, xn.y);
        if (d.x3) d.x3[row] = split3(xn.x, xn.y);
    }
    if (threadIdx.x == 0) {
        d.steps[s] = k + 1;
        d.rms[s] = rms;
    }
}

// Sum over the problem's rows of f(row), block-reduced (deterministic).
#define TC_ROWS(p) for (int64_t rl = threadIdx.x; rl < (p).m; rl += kUpd)

// L-BFGS of one problem with many rows (grid-wide launches, below).  The
// iteration is the host statement's: pair test and store, stop test, two-loop
// recursion (Nocedal & Wright, Alg. 7.4) with H0 = gamma I, descent check,
// max-displacement scaling.  Launched over the grid, each inner product the
// recursion takes with its running vector would be a launch of its own; here
// the recursion is evaluated through inner products instead: each such
// product is expanded into products of the gradient with the stored pairs
// (s_j.g, y_j.g) and of the stored pairs with each other (s_a.y_b, y_a.y_b,
// kept per ring slot and computed once, when the newer of the two pairs is
// stored).  A step then needs one round of reductions over the rows (a pass
// per four stored pairs, all independent) instead of 2 h + 2 that wait on one
// another, and the direction is one combination
// d = c_g g + sum_j (c_s[j] s_j + c_y[j] y_j).  The two forms agree to
// rounding.  (One CTA per problem, k_update_lbfgs, keeps the plain two-loop
// recursion: its reductions are cheap within a CTA, and the expanded form's
// extra float64 products cost more there.)

constexpr int kLbSlotsPerPass = 4;                              // stored pairs per dot pass
constexpr int kLbVals = 6 + 5 * kLbSlotsPerPass;                // values reduced per pass
constexpr int kLbPasses = (kMaxMem + kLbSlotsPerPass - 1) / kLbSlotsPerPass;
constexpr int kLbGram = 2 * kMaxMem * kMaxMem;                  // per problem: s_a.y_b, y_a.y_b by slot

__device__ __forceinline__ int lb_slot(int head, int i, int mem) { return ((head - 1 - i) % mem + mem) % mem; }

// Coefficients of one step of one problem.
struct LbCoef {
    double cg;                         // d = cg gz + sum_j cs[j] S_j + cy[j] Y_j (j: ring slot)
    double cs[kMaxMem], cy[kMaxMem];
    double rms;
    int keep, slot;                    // store the new pair in ring slot `slot`
    int stop;                          // 1: no step (stopped, or measuring)
    int reset;                         // descent check failed: d = -step0 gz
    int hist, head;                    // history after this step's store
};

// The reduced inner products of one step: base[0..5] = gz.gz, s.y, s.s, y.y,
// s.gz, y.gz of the new pair (s = z - z_prev, y = gz - gz_prev); per stored
// pair of age i (0 the newest): S_i.gz, Y_i.gz, s.Y_i, S_i.y, y.Y_i.
struct LbDots {
    double base[6];
    double sg[kMaxMem], yg[kMaxMem], sY[kMaxMem], Sy[kMaxMem], yY[kMaxMem];
};

// One row's share of dot pass `pass`.
__device__ __forceinline__ void lb_row_dots(const RelaxDev& d, int64_t row, int pass, int k, int hist, int head,
                                            int mem, double (&acc)[kLbVals])
{
    const double2 z = d.z[row], gz = d.q[row];
    double2 sn = make_double2(0.0, 0.0), yn = make_double2(0.0, 0.0);
    if (k > 0) {
        const double2 zo = d.xp[row], go = d.gp[row];
        sn = make_double2(z.x - zo.x, z.y - zo.y);
        yn = make_double2(gz.x - go.x, gz.y - go.y);
    }
    if (pass == 0) {
        acc[0] += gz.x * gz.x + gz.y * gz.y;
        acc[1] += sn.x * yn.x + sn.y * yn.y;
        acc[2] += sn.x * sn.x + sn.y * sn.y;
        acc[3] += yn.x * yn.x + yn.y * yn.y;
        acc[4] += sn.x * gz.x + sn.y * gz.y;
        acc[5] += yn.x * gz.x + yn.y * gz.y;
    }
#pragma unroll
    for (int t = 0; t < kLbSlotsPerPass; ++t) {
        const int i = pass * kLbSlotsPerPass + t;
        if (i >= hist) break;
        const int j = lb_slot(head, i, mem);
        const double2 S = d.Sh[(int64_t)j * d.M + row], Y = d.Yh[(int64_t)j * d.M + row];
        acc[6 + 5 * t + 0] += S.x * gz.x + S.y * gz.y;
        acc[6 + 5 * t + 1] += Y.x * gz.x + Y.y * gz.y;
        acc[6 + 5 * t + 2] += sn.x * Y.x + sn.y * Y.y;
        acc[6 + 5 * t + 3] += S.x * yn.x + S.y * yn.y;
        acc[6 + 5 * t + 4] += yn.x * Y.x + yn.y * Y.y;
    }
}

// Scatter the reduced values of pass `pass` into LbDots.
__device__ __forceinline__ void lb_take(LbDots& o, const double* v, int pass)
{
    if (pass == 0)
        for (int c = 0; c < 6; ++c) o.base[c] = v[c];
    for (int t = 0; t < kLbSlotsPerPass; ++t) {
        const int i = pass * kLbSlotsPerPass + t;
        if (i >= kMaxMem) break;
        o.sg[i] = v[6 + 5 * t + 0];
        o.yg[i] = v[6 + 5 * t + 1];
        o.sY[i] = v[6 + 5 * t + 2];
        o.Sy[i] = v[6 + 5 * t + 3];
        o.yY[i] = v[6 + 5 * t + 4];
    }
}

// Problem s's slot products and 1/(s.y) between global memory and a block's
// shared copy (every thread of the block takes part).
__device__ __forceinline__ void lb_gram_load(const RelaxDev& d, int s, double* SY, double* YY, double* rho)
{
    const double* g = d.gram + (int64_t)s * kLbGram;
    for (int e = threadIdx.x; e < kMaxMem * kMaxMem; e += blockDim.x) {
        SY[e] = g[e];
        YY[e] = g[kMaxMem * kMaxMem + e];
    }
    if (threadIdx.x < kMaxMem) rho[threadIdx.x] = d.rho[(int64_t)s * kMaxMem + threadIdx.x];
}

__device__ __forceinline__ void lb_gram_store(RelaxDev& d, int s, const double* SY, const double* YY, const double* rho)
{
    double* g = d.gram + (int64_t)s * kLbGram;
    for (int e = threadIdx.x; e < kMaxMem * kMaxMem; e += blockDim.x) {
        g[e] = SY[e];
        g[kMaxMem * kMaxMem + e] = YY[e];
    }
    if (threadIdx.x < kMaxMem) d.rho[(int64_t)s * kMaxMem + threadIdx.x] = rho[threadIdx.x];
}

// The scalar part of the step (one thread): pair test and store into the
// slot products, stop test, the recursion on inner products, descent check.
// SY, YY, rho: shared-memory copies of problem s's s_a.y_b and y_a.y_b by ring
// slot ([a][b]) and 1/(s_j.y_j) (lb_gram_load / lb_gram_store move them), so
// the dependent chain of the recursion reads no global memory.  Writes hist,
// head, rms, active of problem s.
__device__ void lb_scalars(RelaxDev& d, int s, const Prob& p, const StepParams& sp, const LbDots& t, LbCoef& c,
                           double* SY, double* YY, double* rho)
{
    const int k = d.steps[s], mem = sp.memory;
    const int hist0 = d.hist[s], head0 = d.head[s];
    c.rms = sqrt(t.base[0] / (double)max(p.m, 1));
    c.keep = 0;
    c.slot = head0;
    c.stop = 1;
    c.reset = 0;
    c.hist = hist0;
    c.head = head0;
    if (sp.measure) {
        d.rms[s] = c.rms;
        return;
    }
    // s_j.gz and y_j.gz by ring slot
    double sg[kMaxMem], yg[kMaxMem];
    for (int i = 0; i < hist0; ++i) {
        const int j = lb_slot(head0, i, mem);
        sg[j] = t.sg[i];
        yg[j] = t.yg[i];
    }
    int hist = hist0, head = head0;
    c.keep = k > 0 && t.base[1] > 1e-12 * sqrt(t.base[2]) * sqrt(t.base[3]);
    if (c.keep) {
        const int jn = head0;
        for (int i = 0; i < hist0; ++i) {
            const int j = lb_slot(head0, i, mem);
            if (j == jn) continue;  // the oldest pair, overwritten by the new one
            SY[jn * kMaxMem + j] = t.sY[i];
            SY[j * kMaxMem + jn] = t.Sy[i];
            YY[jn * kMaxMem + j] = YY[j * kMaxMem + jn] = t.yY[i];
        }
        SY[jn * kMaxMem + jn] = t.base[1];
        YY[jn * kMaxMem + jn] = t.base[3];
        rho[jn] = 1.0 / t.base[1];
        sg[jn] = t.base[4];
        yg[jn] = t.base[5];
        head = (head0 + 1) % mem;
        hist = min(hist0 + 1, mem);
    }
    c.hist = hist;
    c.head = head;
    d.rms[s] = c.rms;
    d.hist[s] = hist;
    d.head[s] = head;
    if (sp.gtol > 0.0 && c.rms < sp.gtol) {
        d.active[s] = 0;
        return;
    }
    c.stop = 0;
    // first loop, newest pair first: alpha_i = rho_i s_i.q_i, q_i = gz - sum_{i' < i} alpha_i' y_i'
    double al[kMaxMem], be[kMaxMem];
    int js[kMaxMem];
    for (int i = 0; i < hist; ++i) {
        const int j = lb_slot(head, i, mem);
        js[i] = j;
        double sq = sg[j];
        for (int i2 = 0; i2 < i; ++i2) sq -= al[i2] * SY[j * kMaxMem + js[i2]];
        al[i] = rho[j] * sq;
    }
    const double gamma = hist > 0 ? SY[js[0] * kMaxMem + js[0]] / YY[js[0] * kMaxMem + js[0]] : sp.step0;
    // second loop, oldest pair first: r = gamma q + sum_{older i'} (alpha_i' - beta_i') s_i',
    // beta_i = rho_i y_i.r
    for (int i = hist - 1; i >= 0; --i) {
        const int j = js[i];
        double yq = yg[j];
        for (int i2 = 0; i2 < hist; ++i2) yq -= al[i2] * YY[j * kMaxMem + js[i2]];
        double yr = gamma * yq;
        for (int i2 = hist - 1; i2 > i; --i2) yr += (al[i2] - be[i2]) * SY[js[i2] * kMaxMem + j];
        be[i] = rho[j] * yr;
    }
    // d = -r = -gamma gz + gamma sum alpha_i y_i - sum (alpha_i - beta_i) s_i
    for (int j = 0; j < kMaxMem; ++j) c.cs[j] = c.cy[j] = 0.0;
    c.cg = -gamma;
    double gd = -gamma * t.base[0];
    for (int i = 0; i < hist; ++i) {
        c.cy[js[i]] = gamma * al[i];
        c.cs[js[i]] = -(al[i] - be[i]);
        gd += c.cy[js[i]] * yg[js[i]] + c.cs[js[i]] * sg[js[i]];
    }
    if (gd >= 0.0) {
        c.reset = 1;
        c.hist = c.head = 0;
        d.hist[s] = 0;
        d.head[s] = 0;
        c.cg = -sp.step0;
        for (int j = 0; j < kMaxMem; ++j) c.cs[j] = c.cy[j] = 0.0;
    }
}

// Store the kept pair, keep dE/dz as the previous gradient, and (unless the
// problem stops) write the direction into q; returns |d| of the row.
__device__ __forceinline__ double lb_row_dir(RelaxDev& d, int64_t row, int k, const LbCoef& c, int mem)
{
    const double2 gz = d.q[row];
    if (c.keep) {
        const double2 z = d.z[row], zo = d.xp[row], go = d.gp[row];
        d.Sh[(int64_t)c.slot * d.M + row] = make_double2(z.x - zo.x, z.y - zo.y);
        d.Yh[(int64_t)c.slot * d.M + row] = make_double2(gz.x - go.x, gz.y - go.y);
    }
    d.gp[row] = gz;
    if (c.stop) return 0.0;
    double2 dv = make_double2(c.cg * gz.x, c.cg * gz.y);
    for (int i = 0; i < c.hist; ++i) {
        const int j = lb_slot(c.head, i, mem);
        const double2 S = d.Sh[(int64_t)j * d.M + row], Y = d.Yh[(int64_t)j * d.M + row];
        dv.x += c.cs[j] * S.x + c.cy[j] * Y.x;
        dv.y += c.cs[j] * S.y + c.cy[j] * Y.y;
    }
    d.q[row] = dv;
    return sqrt(dv.x * dv.x + dv.y * dv.y);
}

// The step z <- z + alpha d of one row, then x and its splits.
__device__ __forceinline__ void lb_row_step(RelaxDev& d, int64_t row, double alpha, const StepParams& sp)
{
    const bool pinned = d.flags && d.flags[d.gidx[row]];
    const double2 z = d.z[row], dv = d.q[row];
    d.xp[row] = z;
    if (d.xold) d.xold[row] = d.x[row];
    const double2 zn = make_double2(z.x + alpha * dv.x, z.y + alpha * dv.y);
    d.z[row] = zn;
    const double2 xn = z_to_x(zn, sp.radius, pinned, d.tu);
    d.x[row] = xn;
    d.xs[row] = split4(xn.x, xn.y);
    if (d.x3) d.x3[row] = split3(xn.x, xn.y);
}

// Deterministic block sums of N doubles per thread: a shuffle tree per warp,
// then the warps' partials in warp order.
template <int N> __device__ void block_sums_n(double (&v)[N], double (*red)[N])
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        double x = v[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[w][i] = x;
    }
    __syncthreads();
    if (threadIdx.x < N) {
        double t = red[0][threadIdx.x];
        for (int q = 1; q < kUpd / 32; ++q) t += red[q][threadIdx.x];
        red[0][threadIdx.x] = t;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = red[0][i];
    __syncthreads();
}

// L-BFGS on the wall parameterisation, one CTA per problem (or a queue of problems
// taken by persistent CTAs, k_update_lbfgs).  Same iteration as
// the host statement: pair test and store, stop test, two-loop recursion
// (Nocedal & Wright, Alg. 7.4), descent check, max-displacement scaling.
__device__ void lbfgs_one(const RelaxDev& d, const double2* __restrict__ part_g, const SlotView& v,
                          const StepParams& sp, const int s, double* sh, double* al)
{
    if (!d.active[s]) return;
    const Prob p = d.prob[s];
    if (p.m > kLargeRows) return;  // updated by the grid-wide sequence below
    const int k = d.steps[s];
    const int mem = sp.memory;
    const int64_t M = d.M;
    double* rho = d.rho + (int64_t)s * kMaxMem;
    // new dE/dz into q; pair statistics against the previous z (xp) and dE/dz (gp)
    double acc[4] = {0.0, 0.0, 0.0, 0.0};  // |gzn|^2, s.y, s.s, y.y
    bool bad = false;
    TC_ROWS(p)
    {
        const int64_t row = p.row_base + rl;
        double2 g = sum_g(p, rl, part_g, v);
        if (!isfinite(g.x) || !isfinite(g.y)) bad = true;
        const bool pinned = d.flags && d.flags[d.gidx[row]];
        const double2 z = d.z[row];
        double2 gz = grad_z(z, g, sp.radius, pinned, d.tu);
        d.q[row] = gz;
        acc[0] += gz.x * gz.x + gz.y * gz.y;
        if (k > 0) {
            double2 zo = d.xp[row], go = d.gp[row];
            double sx = z.x - zo.x, sy = z.y - zo.y, yx = gz.x - go.x, yy = gz.y - go.y;
            acc[1] += sx * yx + sy * yy;
            acc[2] += sx * sx + sy * sy;
            acc[3] += yx * yx + yy * yy;
        }
    }
    if (bad) set_status(d.st, ST_NONFINITE);
    block_sums(acc, sh);
    if (sp.measure) {
        if (threadIdx.x == 0) d.rms[s] = sqrt(acc[0] / (double)max(p.m, 1));
        return;
    }
    int hist = d.hist[s], head = d.head[s];
    const bool keep = k > 0 && acc[1] > 1e-12 * sqrt(acc[2]) * sqrt(acc[3]);
    TC_ROWS(p)
    {
        const int64_t row = p.row_base + rl;
        const double2 gz = d.q[row];
        if (keep) {
            const double2 z = d.z[row], zo = d.xp[row], go = d.gp[row];
            d.Sh[(int64_t)head * M + row] = make_double2(z.x - zo.x, z.y - zo.y);
            d.Yh[(int64_t)head * M + row] = make_double2(gz.x - go.x, gz.y - go.y);
        }
        d.gp[row] = gz;
    }
    if (keep) {
        if (threadIdx.x == 0) rho[head] = 1.0 / acc[1];
        head = (head + 1) % mem;
        hist = min(hist + 1, mem);
    }
    const double rms = sqrt(acc[0] / (double)max(p.m, 1));
    if (sp.gtol > 0.0 && rms < sp.gtol) {
        if (threadIdx.x == 0) {
            d.active[s] = 0;
            d.rms[s] = rms;
            d.hist[s] = hist;
            d.head[s] = head;
        }
        return;
    }
    __syncthreads();
    // two-loop recursion on q = dE/dz
    for (int i = 0; i < hist; ++i) {
        const int j = ((head - 1 - i) % mem + mem) % mem;
        double a[1] = {0.0};
        TC_ROWS(p)
        {
            const int64_t row = p.row_base + rl;
            double2 sj = d.Sh[(int64_t)j * M + row], qq = d.q[row];
            a[0] += sj.x * qq.x + sj.y * qq.y;
        }
        block_sums(a, sh);
        const double aj = rho[j] * a[0];
        if (threadIdx.x == 0) al[j] = aj;
        TC_ROWS(p)
        {
            const int64_t row = p.row_base + rl;
            double2 yj = d.Yh[(int64_t)j * M + row], qq = d.q[row];
            d.q[row] = make_double2(qq.x - aj * yj.x, qq.y - aj * yj.y);
        }
        __syncthreads();
    }
    double gamma = sp.step0;
    if (hist > 0) {
        const int j = ((head - 1) % mem + mem) % mem;
        double a[2] = {0.0, 0.0};
        TC_ROWS(p)
        {
            const int64_t row = p.row_base + rl;
            double2 sj = d.Sh[(int64_t)j * M + row], yj = d.Yh[(int64_t)j * M + row];
            a[0] += sj.x * yj.x + sj.y * yj.y;
            a[1] += yj.x * yj.x + yj.y * yj.y;
        }
        block_sums(a, sh);
        gamma = a[0] / a[1];
    }
    TC_ROWS(p)
    {
        const int64_t row = p.row_base + rl;
        double2 qq = d.q[row];
        d.q[row] = make_double2(qq.x * gamma, qq.y * gamma);
    }
    __syncthreads();
    for (int i = hist - 1; i >= 0; --i) {
        const int j = ((head - 1 - i) % mem + mem) % mem;
        double b[1] = {0.0};
        TC_ROWS(p)
        {
            const int64_t row = p.row_base + rl;
            double2 yj = d.Yh[(int64_t)j * M + row], qq = d.q[row];
            b[0] += yj.x * qq.x + yj.y * qq.y;
        }
        block_sums(b, sh);
        const double c = al[j] - rho[j] * b[0];
        TC_ROWS(p)
        {
            const int64_t row = p.row_base + rl;
            double2 sj = d.Sh[(int64_t)j * M + row], qq = d.q[row];
            d.q[row] = make_double2(qq.x + sj.x * c, qq.y + sj.y * c);
        }
        __syncthreads();
    }
    // d = -q; descent check against dE/dz (gp)
    double dd[1] = {0.0};
    TC_ROWS(p)
    {
        const int64_t row = p.row_base + rl;
        double2 qq = d.q[row], gz = d.gp[row];
        dd[0] -= gz.x * qq.x + gz.y * qq.y;
    }
    block_sums(dd, sh);
    const bool reset = dd[0] >= 0.0;
    if (reset) {
        hist = 0;
        head = 0;
    }
    double dmax = 0.0;
    TC_ROWS(p)
    {
        const int64_t row = p.row_base + rl;
        double2 qq = d.q[row], gz = d.gp[row];
        double2 dv = reset ? make_double2(-sp.step0 * gz.x, -sp.step0 * gz.y) : make_double2(-qq.x, -qq.y);
        d.q[row] = dv;
        dmax = fmax(dmax, sqrt(dv.x * dv.x + dv.y * dv.y));
    }
    dmax = block_max(dmax, sh);
    const double alpha = dmax > sp.maxstep ? sp.maxstep / dmax : 1.0;
    if (threadIdx.x == 0 && d.ls_alpha) d.ls_alpha[s] = alpha;
    TC_ROWS(p)
    {
        const int64_t row = p.row_base + rl;
        const bool pinned = d.flags && d.flags[d.gidx[row]];
        double2 z = d.z[row], dv = d.q[row];
        d.xp[row] = z;
        if (d.xold) d.xold[row] = d.x[row];
        double2 zn = make_double2(z.x + alpha * dv.x, z.y + alpha * dv.y);
        d.z[row] = zn;
        double2 xn = z_to_x(zn, sp.radius, pinned, d.tu);
        d.x[row] = xn;
        d.xs[row] = split4(xn.x, xn.y);
        if (d.x3) d.x3[row] = split3(xn.x, xn.y);
    }
    if (threadIdx.x == 0) {
        d.steps[s] = k + 1;
        d.rms[s] = rms;
        d.hist[s] = hist;
        d.head[s] = head;
    }
}

// One CTA per problem (d.upd_order null), or persistent CTAs that take the
// problems of d.upd_order (largest first) from a queue: a ticket counter that
// the CTA drawing the last ticket of the launch sets back to zero.  Each
// problem is stepped by one CTA either way, with the same sums in the same
// order, so the schedule never changes a result.
__global__ void __launch_bounds__(kUpd) k_update_lbfgs(RelaxDev d, const double2* __restrict__ part_g, SlotView v,
                                                        StepParams sp)
{
    __shared__ double sh[kUpd];
    __shared__ double al[kMaxMem];
    __shared__ unsigned ticket;
    if (!d.upd_order) {
        lbfgs_one(d, part_g, v, sp, blockIdx.x, sh, al);
        return;
    }
    for (;;) {
        if (threadIdx.x == 0) ticket = atomicAdd(d.upd_ctr, 1u);
        __syncthreads();
        const unsigned t = ticket;
        __syncthreads();
        if (t >= (unsigned)d.upd_n) {
            // every CTA draws exactly one ticket >= upd_n; the last of them is drawn last
            if (threadIdx.x == 0 && t == (unsigned)d.upd_n + gridDim.x - 1) *d.upd_ctr = 0u;
            return;
        }
        lbfgs_one(d, part_g, v, sp, d.upd_order[t], sh, al);
        __syncthreads();
    }
}

#include "tc_lbfgsb.cuh"

// CTAs per problem of the L-BFGS-B update: the largest cluster size of 16
// (a non-portable size, where the device allows it), 8, 4, 2 that the device
// can run for this kernel and that keeps all problems in one wave
// (problems x size <= SMs), else 1.  A problem's float64 sums are added in an
// order that depends on that size, so its result is deterministic for a given
// number of problems in the call (and bit for bit the same run to run).
template <int CL> static bool lbfgsb_cluster_ok()
{
    if (CL > 8 && cudaFuncSetAttribute(k_update_lbfgsb<CL>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                      cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL);
    cfg.blockDim = dim3(kUpd);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    const cudaError_t e = cudaOccupancyMaxActiveClusters(&n, k_update_lbfgsb<CL>, &cfg);
    if (e != cudaSuccess) cudaGetLastError();
    return e == cudaSuccess && n >= 1;
}

// Largest usable cluster size on the current device (queried once per device).
static int lbfgsb_cluster_max()
{
    static int cached[64];
    static bool known[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return 1;
    }
    if (!known[dev]) {
        cached[dev] = lbfgsb_cluster_ok<16>() ? 16
                      : lbfgsb_cluster_ok<8>() ? 8
                      : lbfgsb_cluster_ok<4>() ? 4
                      : lbfgsb_cluster_ok<2>() ? 2
                                               : 1;
        known[dev] = true;
    }
    return cached[dev];
}

static int lbfgsb_cluster_size(int n_problems)
{
    int c = lbfgsb_cluster_max();
    while (c > 1 && (int64_t)n_problems * c > sm_count()) c /= 2;
    return c;
}

template <int CL>
static cudaError_t launch_lbfgsb_cl(const RelaxDev& d, const double2* part_g, const SlotView& v, const StepParams& sp,
                                    cudaStream_t st)
{
    if constexpr (CL == 1) {
        k_update_lbfgsb<1><<<d.S, kUpd, 0, st>>>(d, part_g, v, sp);
        return cudaGetLastError();
    } else {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)d.S * CL);
        cfg.blockDim = dim3(kUpd);
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = CL;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, k_update_lbfgsb<CL>, d, part_g, v, sp);
    }
}

static cudaError_t launch_lbfgsb(const RelaxDev& d, const double2* part_g, const SlotView& v, const StepParams& sp,
                                 cudaStream_t st)
{
    switch (lbfgsb_cluster_size(d.S)) {
        case 16: return launch_lbfgsb_cl<16>(d, part_g, v, sp, st);
        case 8: return launch_lbfgsb_cl<8>(d, part_g, v, sp, st);
        case 4: return launch_lbfgsb_cl<4>(d, part_g, v, sp, st);
        case 2: return launch_lbfgsb_cl<2>(d, part_g, v, sp, st);
        default: return launch_lbfgsb_cl<1>(d, part_g, v, sp, st);
    }
}

// ------------------------------------------- L-BFGS for large problems ---
// The same step as k_update_lbfgs for one problem with many rows, as a fixed
// sequence of grid-wide launches: the dot passes (per-block partials), one
// thread for the scalars (partials added in block order, so the result does
// not depend on scheduling), the direction (per-block maxima of |d|) and the
// step.  No launch waits on another CTA.

struct LbArgs {
    int s;
    double* part;  // [kLbPasses][kLargeBlocks][kLbVals]
    LbCoef* c;
};

#define TC_GRID_ROWS(p) for (int64_t rl = blockIdx.x * (int64_t)kUpd + threadIdx.x; rl < (p).m; rl += (int64_t)gridDim.x * kUpd)

// Dot pass `pass` (pass 0 also forms dE/dz into q).
__global__ void __launch_bounds__(kUpd) k_lb_dots(RelaxDev d, LbArgs la, const double2* __restrict__ part_g,
                                                  SlotView v, StepParams sp, int pass)
{
    __shared__ double red[kUpd / 32][kLbVals];
    if (!d.active[la.s]) return;
    const Prob p = d.prob[la.s];
    const int k = d.steps[la.s], hist0 = sp.measure ? 0 : d.hist[la.s], head0 = d.head[la.s];
    if (pass > 0 && pass * kLbSlotsPerPass >= hist0) return;
    bool bad = false;
    double acc[kLbVals];
#pragma unroll
    for (int q = 0; q < kLbVals; ++q) acc[q] = 0.0;
    TC_GRID_ROWS(p)
    {
        const int64_t row = p.row_base + rl;
        if (pass == 0) {
            const double2 g = sum_g(p, rl, part_g, v);
            if (!isfinite(g.x) || !isfinite(g.y)) bad = true;
            const bool pinned = d.flags && d.flags[d.gidx[row]];
            d.q[row] = grad_z(d.z[row], g, sp.radius, pinned, d.tu);
        }
        lb_row_dots(d, row, pass, k, hist0, head0, sp.memory, acc);
    }
    if (bad) set_status(d.st, ST_NONFINITE);
    block_sums_n<kLbVals>(acc, red);
    if (threadIdx.x < kLbVals)
        la.part[((int64_t)pass * kLargeBlocks + blockIdx.x) * kLbVals + threadIdx.x] = red[0][threadIdx.x];
}

// The scalars: the partials of every pass added in block order (one column
// per thread), then the scalar step on thread 0 from shared copies.
__global__ void __launch_bounds__(kUpd) k_lb_scalars(RelaxDev d, LbArgs la, StepParams sp)
{
    __shared__ double tv[kLbPasses][kLbVals];
    __shared__ double sSY[kMaxMem * kMaxMem], sYY[kMaxMem * kMaxMem], srho[kMaxMem];
    __shared__ LbDots tot;
    LbCoef& c = *la.c;
    if (!d.active[la.s]) {
        if (threadIdx.x == 0) {
            c.keep = 0;
            c.stop = 1;
            c.hist = -1;  // inactive on entry: the direction and step launches do nothing
        }
        return;
    }
    const Prob p = d.prob[la.s];
    const int hist0 = sp.measure ? 0 : d.hist[la.s];
    const int passes = max(1, (hist0 + kLbSlotsPerPass - 1) / kLbSlotsPerPass);
    for (int e = threadIdx.x; e < passes * kLbVals; e += blockDim.x) {
        const int pass = e / kLbVals, q = e % kLbVals;
        double t = 0.0;
        for (int b = 0; b < kLargeBlocks; ++b) t += la.part[((int64_t)pass * kLargeBlocks + b) * kLbVals + q];
        tv[pass][q] = t;
    }
    lb_gram_load(d, la.s, sSY, sYY, srho);
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int pass = 0; pass < passes; ++pass) lb_take(tot, tv[pass], pass);
        lb_scalars(d, la.s, p, sp, tot, c, sSY, sYY, srho);
    }
    __syncthreads();
    if (!sp.measure) lb_gram_store(d, la.s, sSY, sYY, srho);
}

// Pair store, previous gradient, direction; per-block maximum of |d|.
__global__ void __launch_bounds__(kUpd) k_lb_dir(RelaxDev d, LbArgs la, StepParams sp)
{
    __shared__ double sh[kUpd];
    const LbCoef& c = *la.c;
    if (sp.measure || c.hist < 0) return;
    const Prob p = d.prob[la.s];
    const int k = d.steps[la.s];
    double mx = 0.0;
    TC_GRID_ROWS(p) mx = fmax(mx, lb_row_dir(d, p.row_base + rl, k, c, sp.memory));
    mx = block_max(mx, sh);
    if (threadIdx.x == 0) la.part[blockIdx.x] = mx;
}

// The step; every block takes the maximum over the blocks' maxima in block order.
__global__ void __launch_bounds__(kUpd) k_lb_step(RelaxDev d, LbArgs la, StepParams sp)
{
    const LbCoef& c = *la.c;
    if (c.hist < 0 || c.stop) return;
    const Prob p = d.prob[la.s];
    double dmax = 0.0;
    for (int b = 0; b < kLargeBlocks; ++b) dmax = fmax(dmax, la.part[b]);
    const double alpha = dmax > sp.maxstep ? sp.maxstep / dmax : 1.0;
    TC_GRID_ROWS(p) lb_row_step(d, p.row_base + rl, alpha, sp);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (d.ls_alpha) d.ls_alpha[la.s] = alpha;
        d.steps[la.s] = d.steps[la.s] + 1;
    }
}

// Launches of one step of one large problem (measure: the RMS only).
static int lbfgs_large_launches(const StepParams& sp)
{
    return sp.measure ? 2 : (sp.memory + kLbSlotsPerPass - 1) / kLbSlotsPerPass + 3;
}

static cudaError_t lbfgs_large(RelaxDev& d, LbArgs la, const double2* part_g, SlotView v, const StepParams& sp,
                               cudaStream_t s)
{
    const int passes = sp.measure ? 1 : std::max(1, (sp.memory + kLbSlotsPerPass - 1) / kLbSlotsPerPass);
    for (int pass = 0; pass < passes; ++pass) k_lb_dots<<<kLargeBlocks, kUpd, 0, s>>>(d, la, part_g, v, sp, pass);
    k_lb_scalars<<<1, kUpd, 0, s>>>(d, la, sp);
    if (!sp.measure) {
        k_lb_dir<<<kLargeBlocks, kUpd, 0, s>>>(d, la, sp);
        k_lb_step<<<kLargeBlocks, kUpd, 0, s>>>(d, la, sp);
    }
    return cudaGetLastError();
}

// ----------------------------------------------------- energy changes ---

__global__ void k_rows4(RelaxDev d, const double2* __restrict__ newpos)
{
    for (int64_t rr = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; rr < d.M; rr += (int64_t)gridDim.x * blockDim.x) {
        double2 o = d.pos[d.gidx[rr]];
        double2 nw = newpos[rr];
        d.rows4[rr] = make_d4(o.x, o.y, nw.x, nw.y);
    }
}

// Rows of the difference-form pass: old position split hi/lo and the move
// new - old (rounded once to float32).
__global__ void k_rows8(RelaxDev d, const double2* __restrict__ newpos, f8* __restrict__ rows8)
{
    for (int64_t rr = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; rr < d.M; rr += (int64_t)gridDim.x * blockDim.x) {
        const double2 o = d.pos[d.gidx[rr]];
        const double2 nw = newpos[rr];
        if (!isfinite(nw.x) || !isfinite(nw.y)) set_status(d.st, ST_NONFINITE);
        rows8[rr] = make_f8(split4(o.x, o.y), (float)(nw.x - o.x), (float)(nw.y - o.y));
    }
}

// ---- Armijo backtracking for the L-BFGS step (prm->line_search halvings) ----
// After an L-BFGS update has placed problem s at the trial z = z_k + alpha d
// (z_k in xp, d in q, x before the step in xold), the energy change of the
// move is computed as pair differences (float64, or the float32 difference
// form in the mixed phase) and the trial kept once
//     E(x(z)) - E(x(z_k)) <= 1e-4 alpha (dE/dz . d);
// otherwise alpha is halved and the rows move again.  The last trial is kept.

// Per problem: dE/dz . d of the step just proposed; the problem is tested iff
// it stepped.
__global__ void __launch_bounds__(kUpd) k_ls_begin(RelaxDev d)
{
    __shared__ double sh[kUpd];
    const int s = blockIdx.x;
    const bool stepped = d.active[s] != 0;
    if (!stepped) {
        if (threadIdx.x == 0) d.ls_active[s] = 0;
        return;
    }
    const Prob p = d.prob[s];
    double gd = 0.0;
    TC_ROWS(p)
    {
        const int64_t row = p.row_base + rl;
        const double2 gz = d.gp[row], dv = d.q[row];
        gd += gz.x * dv.x + gz.y * dv.y;
    }
    gd = block_sum<kUpd>(gd, sh);
    if (threadIdx.x == 0) {
        d.ls_gd[s] = gd;
        d.ls_active[s] = 1;
    }
}

// Rows of the energy-change pass for the problems still testing a trial.
__global__ void k_ls_rows(RelaxDev d, int mixed)
{
    for (int64_t rr = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; rr < d.M; rr += (int64_t)gridDim.x * blockDim.x) {
        const int s = find_row_prob(d.prob, d.S, rr);
        if (!d.ls_active[s]) continue;
        const double2 o = d.xold[rr], nw = d.x[rr];
        if (mixed)
            d.rows8[rr] = make_f8(split4(o.x, o.y), (float)(nw.x - o.x), (float)(nw.y - o.y));
        else
            d.rows4[rr] = make_d4(o.x, o.y, nw.x, nw.y);
    }
}

// Armijo test of problem s (one CTA per problem); a failed test halves alpha.
__global__ void __launch_bounds__(kUpd) k_ls_check(RelaxDev d, const double* __restrict__ part_e, SlotView v, int last)
{
    __shared__ double sh[kUpd];
    const int s = blockIdx.x;
    if (!d.ls_active[s]) return;
    const Prob p = d.prob[s];
    double hi = 0.0, lo = 0.0;
    TC_ROWS(p) dd_add(hi, lo, sum_e(p, rl, part_e, v));
    const double dE = block_sum<kUpd>(hi, sh) + block_sum<kUpd>(lo, sh);
    if (threadIdx.x == 0) {
        const double alpha = d.ls_alpha[s];
        if (!isfinite(dE)) set_status(d.st, ST_NONFINITE);
        if (last || dE <= 1e-4 * alpha * d.ls_gd[s]) {
            d.ls_active[s] = 0;
        } else {
            d.ls_alpha[s] = 0.5 * alpha;
        }
    }
}

// Move the rows of the problems whose trial failed to z_k + alpha d.
__global__ void k_ls_move(RelaxDev d, double radius)
{
    for (int64_t rr = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; rr < d.M; rr += (int64_t)gridDim.x * blockDim.x) {
        const int s = find_row_prob(d.prob, d.S, rr);
        if (!d.ls_active[s]) continue;
        const double alpha = d.ls_alpha[s];
        const bool pinned = d.flags && d.flags[d.gidx[rr]];
        const double2 zk = d.xp[rr], dv = d.q[rr];
        double2 zn = make_double2(zk.x + alpha * dv.x, zk.y + alpha * dv.y);
        if (d.boxed) {
            double2 lo, hi;
            tu_bounds(pinned, lo, hi);
            zn = make_double2(clampd(zn.x, lo.x, hi.x), clampd(zn.y, lo.y, hi.y));
        }
        d.z[rr] = zn;
        const double2 xn = z_to_x(zn, radius, pinned, d.tu);
        d.x[rr] = xn;
        d.xs[rr] = split4(xn.x, xn.y);
        if (d.x3) d.x3[rr] = split3(xn.x, xn.y);
    }
}

// Per problem: the difference-form energy change and its error bound.
// |float32 evaluation - exact| <= 2^-15 sum(b), u = 2^-24: each term is within
// about 25 u b of its exact value (separations from hi/lo differences, moves
// rounded once, two MUFU.RSQ and one MUFU.RCP of at most ~2 ulp, a handful of
// roundings), |term| <= b, and a tile sum of 256 float32 terms adds at most
// 256 u sum |term|; 512 u covers both.  Valid for separations above ~1e-6 (below
// that the absolute 2^-47 error of the lo-part differences is not covered).
__global__ void __launch_bounds__(kUpd) k_dmix_sums(RelaxDev d, const double* __restrict__ part_e,
                                                     const double2* __restrict__ part_b, SlotView v,
                                                     double* __restrict__ out, double* __restrict__ bound)
{
    __shared__ double sh[kUpd];
    const int s = blockIdx.x;
    const Prob p = d.prob[s];
    double hi = 0.0, lo = 0.0, b = 0.0;
    TC_ROWS(p)
    {
        dd_add(hi, lo, sum_e(p, rl, part_e, v));
        b += sum_g(p, rl, part_b, v).x;
    }
    const double t = block_sum<kUpd>(hi, sh) + block_sum<kUpd>(lo, sh);
    b = block_sum<kUpd>(b, sh);
    if (threadIdx.x == 0) {
        out[s] = t;
        if (bound) bound[s] = ldexp(b, -15);
        if (!isfinite(t)) set_status(d.st, ST_NONFINITE);
    }
}

// Per problem: sum of its rows' partials (compensated) into out[s].
__global__ void __launch_bounds__(kUpd) k_problem_sums(RelaxDev d, const double* __restrict__ part_e, SlotView v,
                                                        double* out, const int* __restrict__ only)
{
    __shared__ double sh[kUpd];
    const int s = blockIdx.x;
    if (only && !only[s]) return;
    const Prob p = d.prob[s];
    double hi = 0.0, lo = 0.0;
    TC_ROWS(p) dd_add(hi, lo, sum_e(p, rl, part_e, v));
    double t = block_sum<kUpd>(hi, sh) + block_sum<kUpd>(lo, sh);
    if (threadIdx.x == 0) {
        out[s] = t;
        if (!isfinite(t)) set_status(d.st, ST_NONFINITE);
    }
}

// Sequential accept, problem s: reduce its energy change, apply it if negative,
// then decide whether problem s + 1 is free of accepted charges.
__global__ void __launch_bounds__(kUpd) k_accept_apply(RelaxDev d, int s, const double* __restrict__ part1, SlotView v)
{
    __shared__ double sh[kUpd];
    __shared__ int clash;
    const Prob p = d.prob[s];
    if (d.ok[s]) {
        double hi = 0.0, lo = 0.0;
        TC_ROWS(p) dd_add(hi, lo, sum_e(p, rl, part1, v));
        const double de = block_sum<kUpd>(hi, sh) + block_sum<kUpd>(lo, sh);
        const bool acc = de < 0.0;
        if (!isfinite(de)) set_status(d.st, ST_NONFINITE);
        if (acc) {
            TC_ROWS(p)
            {
                const int64_t row = p.row_base + rl;
                const int32_t j = d.gidx[row];
                d.pos[j] = d.x[row];
                atomicOr(&d.taken[j >> 5], 1u << (j & 31));
            }
        }
        if (threadIdx.x == 0) {
            d.delta[s] = de;
            d.status[s] = acc ? 1 : 0;
        }
    } else if (threadIdx.x == 0) {
        d.delta[s] = 0.0;
        d.status[s] = 2;
    }
    if (s + 1 >= d.S) return;
    __threadfence();
    if (threadIdx.x == 0) clash = 0;
    __syncthreads();
    const Prob q = d.prob[s + 1];
    TC_ROWS(q)
    {
        const int32_t j = d.gidx[q.row_base + rl];
        if ((((volatile uint32_t*)d.taken)[j >> 5] >> (j & 31)) & 1u) clash = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) d.ok[s + 1] = clash ? 0 : 1;
}

// Instance mode write-back: every row (accept = 0) or the rows of problems
// whose energy change is negative (accept = 1).
__global__ void k_write_back(RelaxDev d, int accept)
{
    for (int64_t rr = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; rr < d.M; rr += (int64_t)gridDim.x * blockDim.x) {
        const int s = find_row_prob(d.prob, d.S, rr);
        if (accept && !(d.delta[s] < 0.0)) continue;
        d.pos[d.gidx[rr]] = d.x[rr];
    }
}

__global__ void k_results(RelaxDev d, tc_subdomain_result* out, int mode_instances, int accept, int want_energy)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= d.S) return;
    tc_subdomain_result r;
    r.delta_e = accept ? d.delta[s] : NAN;
    r.energy = want_energy ? d.energy[s] : NAN;
    r.rms = d.rms[s];
    r.steps = d.steps[s];
    if (mode_instances)
        r.status = accept ? (d.delta[s] < 0.0 ? 1 : 0) : 1;
    else
        r.status = accept ? d.status[s] : 0;
    out[s] = r;
}

// ------------------------------------------------------------- driver ---

static tc_status check_params(const tc_relax_params* prm)
{
    if (!prm) return TC_ERR_INVALID_ARG;
    if (prm->precision != TC_FP64 && prm->precision != TC_MIXED && prm->precision != TC_F64X) return TC_ERR_INVALID_ARG;
    if (prm->polish_precision != TC_FP64 && prm->polish_precision != TC_F64X) return TC_ERR_INVALID_ARG;
    if (prm->line_search < 0 || prm->line_search > 30) return TC_ERR_INVALID_ARG;
    if (prm->optimizer < TC_OPT_GD || prm->optimizer > TC_OPT_LBFGSB_TU) return TC_ERR_INVALID_ARG;
    const bool lbfgs = prm->optimizer >= TC_OPT_LBFGS;
    if (prm->optimizer == TC_OPT_LBFGSB_TU && prm->memory > kBMem) {
        set_last_error("tc_relax_subdomains: L-BFGS-B keeps at most 8 pairs");
        return TC_ERR_INVALID_ARG;
    }
    if (prm->n_steps < 0 || prm->polish_steps < 0) return TC_ERR_INVALID_ARG;
    if (lbfgs && (prm->memory < 1 || prm->memory > kMaxMem)) return TC_ERR_INVALID_ARG;
    if (!(prm->radius > 0.0) || !(prm->step0 > 0.0)) return TC_ERR_INVALID_ARG;
    if (prm->optimizer == TC_OPT_BB && !(prm->alpha_max >= prm->alpha_min && prm->alpha_min >= 0.0))
        return TC_ERR_INVALID_ARG;
    if (lbfgs && !(prm->maxstep > 0.0)) return TC_ERR_INVALID_ARG;
    if (!(prm->gtol >= 0.0) || !(prm->polish_gtol >= 0.0)) return TC_ERR_INVALID_ARG;
    return TC_OK;
}

struct Host {
    std::vector<int64_t> off, world;
};

// Launch timing of the last profiled call (per host thread).
thread_local tc_relax_profile g_last_profile{};

// CUDA events of one profiled call, created on demand per device and reused.
struct EventPool {
    std::vector<cudaEvent_t> ev;
    cudaEvent_t get(size_t i)
    {
        while (ev.size() <= i) {
            cudaEvent_t e = nullptr;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            ev.push_back(e);
        }
        return ev[i];
    }
};
thread_local EventPool g_events;

static double elapsed(cudaEvent_t a, cudaEvent_t b)
{
    float ms = 0.f;
    if (!a || !b) return 0.0;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
        cudaGetLastError();  // a timing query failure must not surface at a later launch check
        return 0.0;
    }
    return ms;
}

static_assert(sizeof(tc_subdomain_result) == 32, "tc_subdomain_result layout");
static_assert(sizeof(tc_relax_params) == 96, "tc_relax_params layout");
static_assert(sizeof(tc_relax_profile) == 56, "tc_relax_profile layout");

// One relaxation phase: `steps` x (pass, update), captured into a CUDA graph.
// Problems whose L-BFGS update runs as the grid-wide sequence.
struct LargeSet {
    std::vector<int> ids;
    double* part = nullptr;
    LbCoef* sc = nullptr;  // one per entry of ids
};

// The energy-change pass of the line search: float32 difference form in the
// mixed phase, float64 pair differences otherwise.
struct LsArgs {
    PassArgs a;       // rows: rows8 (mixed) or rows4; active: ls_active
    int64_t G = 1;    // CTAs of that pass
    bool mixed = false;
};

static cudaError_t line_search(RelaxDev& d, const LsArgs& ls, const Plan& P, const StepParams& sp, cudaStream_t s,
                               int& launches)
{
    const int eb = (int)std::max<int64_t>(1, std::min<int64_t>((d.M + 255) / 256, 8L * sm_count()));
    SlotView v{P.W, ls.G, 0, P.M, 0};
    k_ls_begin<<<d.S, kUpd, 0, s>>>(d);
    cudaError_t e = cudaGetLastError();
    for (int t = 0; t < sp.line_search && e == cudaSuccess; ++t) {
        k_ls_rows<<<eb, 256, 0, s>>>(d, ls.mixed ? 1 : 0);
        e = ls.mixed ? launch_pass<PASS_DMIX, false, false>(ls.a, ls.G, 0, 0, s)
                     : launch_pass<PASS_DELTA, false, false>(ls.a, ls.G, 0, 0, s);
        if (e != cudaSuccess) break;
        k_ls_check<<<d.S, kUpd, 0, s>>>(d, ls.a.part_e, v, t == sp.line_search - 1 ? 1 : 0);
        k_ls_move<<<eb, 256, 0, s>>>(d, sp.radius);
        e = cudaGetLastError();
        launches += 4;
    }
    return e;
}

// Steps captured in one CUDA graph and replayed (the last chunk may be shorter).
constexpr int kChunkSteps = 64;

// OR of the problems' active flags, for the host's early stop between chunks.
__global__ void k_any_active(const int* __restrict__ active, int S, int* __restrict__ any)
{
    __shared__ int sh;
    if (threadIdx.x == 0) sh = 0;
    __syncthreads();
    int a = 0;
    for (int k = threadIdx.x; k < S; k += blockDim.x) a |= active[k] != 0;
    if (a) sh = 1;
    __syncthreads();
    if (threadIdx.x == 0) *any = sh;
}

// The launches of one step (pass, optimiser update, line search) on stream st;
// ev_mid (nullable) is recorded between the pass and the update.
template <int KIND>
static cudaError_t launch_step(RelaxDev& d, const PassArgs& a, const Plan& P, int64_t G, const StepParams& sp,
                               cudaStream_t st, int& launches, const LargeSet& large, const LsArgs* ls,
                               cudaEvent_t ev_mid)
{
    SlotView v = pass_view(a, P.W, G, P.M);
    cudaError_t e = launch_pass<KIND, false, true>(a, G, 0, 0, st);
    if (e != cudaSuccess) return e;
    if (sp.pre_reduce && a.W > 0) {
        k_sum_slots<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((P.M + 255) / 256, 8L * sm_count())), 256, 0, st>>>(
            d, a.part_g, v);
        v.red = d.g_red;
        ++launches;
    }
    if (ev_mid && (e = cudaEventRecord(ev_mid, st)) != cudaSuccess) return e;
    if (sp.opt == TC_OPT_LBFGSB_TU) {
        e = launch_lbfgsb(d, a.part_g, v, sp, st);
        if (e == cudaSuccess && ls && sp.line_search > 0) e = line_search(d, *ls, P, sp, st, launches);
    } else if (sp.opt == TC_OPT_LBFGS || sp.opt == TC_OPT_LBFGS_TU) {
        k_update_lbfgs<<<d.upd_order ? d.upd_ctas : d.S, kUpd, 0, st>>>(d, a.part_g, v, sp);
        for (size_t q = 0; q < large.ids.size(); ++q) {
            LbArgs la{large.ids[q], large.part, large.sc + q};
            if (e == cudaSuccess) e = lbfgs_large(d, la, a.part_g, v, sp, st);
            launches += lbfgs_large_launches(sp);
        }
        if (e == cudaSuccess && ls && sp.line_search > 0) e = line_search(d, *ls, P, sp, st, launches);
    } else {
        k_update_gdbb<<<d.S, kUpd, 0, st>>>(d, a.part_g, v, sp);
    }
    launches += (a.W > 0 ? 1 : 0) + 1;
    return e == cudaSuccess ? cudaGetLastError() : e;
}

// One more pass at the final rows and a measuring update: the reported RMS
// describes the returned configuration.
template <int KIND>
static cudaError_t launch_measure(RelaxDev& d, const PassArgs& a, const Plan& P, int64_t G, const StepParams& sp,
                                  cudaStream_t st, int& launches, const LargeSet& large)
{
    SlotView v = pass_view(a, P.W, G, P.M);
    cudaError_t e = launch_pass<KIND, false, true>(a, G, 0, 0, st);
    if (e != cudaSuccess) return e;
    if (sp.pre_reduce && a.W > 0) {
        k_sum_slots<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((P.M + 255) / 256, 8L * sm_count())), 256, 0, st>>>(
            d, a.part_g, v);
        v.red = d.g_red;
        ++launches;
    }
    StepParams sm = sp;
    sm.measure = 1;
    if (sp.opt == TC_OPT_LBFGSB_TU) {
        launch_lbfgsb(d, a.part_g, v, sm, st);
    } else if (sp.opt == TC_OPT_LBFGS || sp.opt == TC_OPT_LBFGS_TU) {
        k_update_lbfgs<<<d.upd_order ? d.upd_ctas : d.S, kUpd, 0, st>>>(d, a.part_g, v, sm);
        for (size_t q = 0; q < large.ids.size(); ++q) {
            LbArgs la{large.ids[q], large.part, large.sc + q};
            lbfgs_large(d, la, a.part_g, v, sm, st);
            launches += lbfgs_large_launches(sm);
        }
    } else {
        k_update_gdbb<<<d.S, kUpd, 0, st>>>(d, a.part_g, v, sm);
    }
    launches += (a.W > 0 ? 1 : 0) + 1;
    return cudaGetLastError();
}

// The step loop of one phase.  Three ways to launch it:
//  - profiled: directly on s, with an event between each pass and update;
//  - inside a caller's stream capture: every step joins the caller's graph;
//  - otherwise: kChunkSteps steps are captured once on a private stream and the
//    graph is replayed on s (the executable graph comes from a per-device cache
//    and is updated in place when an earlier call had the same shape, so a
//    repeated call does not instantiate again); with a stopping tolerance the host checks between
//    replays whether any problem is still active and stops when none is (the
//    steps it skips would have been no-ops: every kernel returns at once for an
//    inactive problem).  A shorter last chunk is launched directly.
template <int KIND>
static tc_status run_phase(RelaxDev& d, PassArgs a, const Plan& P, int64_t G, const StepParams& sp, int steps,
                           cudaStream_t s, bool prof, int& launches, const LargeSet& large,
                           const LsArgs* ls = nullptr)
{
    if (steps <= 0) return TC_OK;
    cudaStreamCaptureStatus cs;
    if (cudaError_t e_ = cudaStreamIsCapturing(s, &cs); e_ != cudaSuccess) return cuda_fail(e_, "cudaStreamIsCapturing");
    cudaError_t e = cudaSuccess;
    const char* where = "step loop launch";
    if (prof) {
        // events 0 .. 2 steps: [pass k] between 2k and 2k+1, [update k] between 2k+1 and 2k+2
        e = cudaEventRecord(g_events.get(0), s);
        for (int k = 0; k < steps && e == cudaSuccess; ++k) {
            e = launch_step<KIND>(d, a, P, G, sp, s, launches, large, ls, g_events.get(2 * k + 1));
            if (e == cudaSuccess) e = cudaEventRecord(g_events.get(2 * k + 2), s);
        }
        if (e == cudaSuccess) e = launch_measure<KIND>(d, a, P, G, sp, s, launches, large);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) {
            for (int k = 0; k < steps; ++k) {
                g_last_profile.pass_ms += elapsed(g_events.get(2 * k), g_events.get(2 * k + 1));
                g_last_profile.update_ms += elapsed(g_events.get(2 * k + 1), g_events.get(2 * k + 2));
            }
            g_last_profile.relax_ms += elapsed(g_events.get(0), g_events.get(2 * steps));
            g_last_profile.n_pass += a.W > 0 ? steps : 0;
        }
        return cuda_status(e, where);
    }
    if (cs != cudaStreamCaptureStatusNone) {
        for (int k = 0; k < steps && e == cudaSuccess; ++k) e = launch_step<KIND>(d, a, P, G, sp, s, launches, large, ls, nullptr);
        if (e == cudaSuccess) e = launch_measure<KIND>(d, a, P, G, sp, s, launches, large);
        return cuda_status(e, where);
    }
    const int K = std::min(steps, kChunkSteps);
    tc_status err = TC_OK;
    cudaStream_t cap = capture_stream(&err);
    if (!cap) return err;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int per_chunk = 0;
    if ((e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    for (int k = 0; k < K && e == cudaSuccess; ++k) e = launch_step<KIND>(d, a, P, G, sp, cap, per_chunk, large, ls, nullptr);
    cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
    if (e == cudaSuccess && (e = e2) != cudaSuccess) where = "cudaStreamEndCapture";
    if (e == cudaSuccess && !(exec = take_graph_exec(graph, &e))) where = "cudaGraphInstantiate";
    int done = 0;
    while (e == cudaSuccess && done + K <= steps) {
        if ((e = cudaGraphLaunch(exec, s)) != cudaSuccess) {
            where = "cudaGraphLaunch";
            break;
        }
        done += K;
        launches += per_chunk;
        if (done < steps && sp.gtol > 0.0) {
            int any = 1;
            k_any_active<<<1, 256, 0, s>>>(d.active, d.S, d.any_active);
            ++launches;
            if ((e = cudaMemcpyAsync(&any, d.any_active, sizeof(int), cudaMemcpyDeviceToHost, s)) == cudaSuccess)
                e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) {
                where = "step loop execution";
                break;
            }
            if (!any) done = steps;  // every problem has stopped
        }
    }
    for (; e == cudaSuccess && done < steps; ++done) e = launch_step<KIND>(d, a, P, G, sp, s, launches, large, ls, nullptr);
    if (e == cudaSuccess) e = launch_measure<KIND>(d, a, P, G, sp, s, launches, large);
    // the executable graph is destroyed only after its launches have finished
    cudaError_t e3 = cudaStreamSynchronize(s);
    if (e == cudaSuccess && (e = e3) != cudaSuccess) where = "step loop execution";
    // a graph that ran cleanly goes back to the cache: the next call of this shape updates it in
    // place (cudaGraphExecUpdate) instead of instantiating a new one
    if (exec && e == cudaSuccess)
        give_graph_exec(exec);
    else if (exec)
        cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    return cuda_status(e, where);
}

tc_status relax(double* pos, int64_t n, const int32_t* idx, const int64_t* offsets, int32_t n_sub,
                       const int64_t* world, const uint8_t* flags, const tc_relax_params* prm,
                       tc_subdomain_result* out, cudaStream_t s)
{
    tc_status err = check_params(prm);
    if (err != TC_OK) return err;
    if (n < 0 || n_sub < 0 || (n > 0 && !pos) || (n_sub > 0 && !out) || (reinterpret_cast<uintptr_t>(pos) & 15) ||
        (reinterpret_cast<uintptr_t>(out) & 7))
        return TC_ERR_INVALID_ARG;
    const bool inst = idx == nullptr;
    if (inst && !world) return TC_ERR_INVALID_ARG;
    if (!inst && !offsets) return TC_ERR_INVALID_ARG;
    g_last_profile = tc_relax_profile{};
    if (n_sub == 0) return TC_OK;
    int* st = device_status(&err);
    if (!st) return err;
    const bool prof = prm->profile != 0;
    int launches = 0;
    cudaEvent_t ev_a = nullptr, ev_b = nullptr, ev_c = nullptr, ev_d = nullptr;
    if (prof) {
        // events 0 .. 2 max_steps belong to run_phase; four more after them
        size_t base = 2 * (size_t)std::max(prm->n_steps, prm->polish_steps) + 2;
        ev_a = g_events.get(base);
        ev_b = g_events.get(base + 1);
        ev_c = g_events.get(base + 2);
        ev_d = g_events.get(base + 3);
        if (!ev_a || !ev_b || !ev_c || !ev_d) return TC_ERR_CUDA;
        // every event is created here: none may be created while a graph is being captured
    }

    // sizes to the host (one synchronisation per call)
    Host h;
    if (!inst) {
        h.off.resize(n_sub + 1);
        if (cudaError_t e_ = cudaMemcpyAsync(h.off.data(), offsets, 8 * (n_sub + 1), cudaMemcpyDeviceToHost, s); e_ != cudaSuccess) return cuda_fail(e_, "cudaMemcpyAsync");
    }
    if (world) {
        h.world.resize(2 * (size_t)n_sub);
        if (cudaError_t e_ = cudaMemcpyAsync(h.world.data(), world, 16 * (size_t)n_sub, cudaMemcpyDeviceToHost, s); e_ != cudaSuccess) return cuda_fail(e_, "cudaMemcpyAsync");
    }
    if (cudaError_t e_ = cudaStreamSynchronize(s); e_ != cudaSuccess) return cuda_fail(e_, "cudaStreamSynchronize");

    Plan P;
    P.prob.resize(n_sub);
    std::vector<int64_t> wbeg(n_sub);
    int64_t rows = 0, mask_words = 0, max_m = 0;
    for (int32_t k = 0; k < n_sub; ++k) {
        int64_t wb = world ? h.world[2 * k] : 0, we = world ? h.world[2 * k + 1] : n;
        if (wb < 0 || we > n || wb > we) return TC_ERR_INVALID_ARG;
        Prob& p = P.prob[k];
        int64_t m;
        if (inst) {
            m = we - wb;
            p.row_base = rows;
            p.snap_b = p.snap_e = 0;
            p.mask_off = -1;
        } else {
            if (h.off[k + 1] < h.off[k] || h.off[0] != 0) return TC_ERR_INVALID_ARG;
            m = h.off[k + 1] - h.off[k];
            if (m > we - wb) return TC_ERR_INVALID_ARG;
            p.row_base = h.off[k];
            p.snap_b = wb;
            p.snap_e = we;
            p.mask_off = mask_words;
            mask_words += (we - wb + 31) / 32;
        }
        if (m > INT32_MAX / 2) return TC_ERR_INVALID_ARG;
        p.m = (int32_t)m;
        wbeg[k] = wb;
        rows += m;
        max_m = std::max(max_m, m);
    }
    if (n > INT32_MAX) return TC_ERR_INVALID_ARG;
    P.M = rows;
    plan_units(P);
    const int prec = prm->precision;
    const bool lbfgs = prm->optimizer >= TC_OPT_LBFGS;
    const bool boxed = prm->optimizer == TC_OPT_LBFGSB_TU;
    if (boxed) (void)lbfgsb_cluster_max();  // queried here, outside any stream capture
    const int mem = lbfgs ? prm->memory : 0;
    const int64_t G_bulk = prec == TC_MIXED  ? pass_grid<PASS_MIXED, false, true>(P.W)
                           : prec == TC_F64X ? pass_grid<PASS_F64X, false, true>(P.W)
                                             : pass_grid<PASS_F64, false, true>(P.W);
    const bool polish_x = prm->polish_precision == TC_F64X;
    const int64_t G_f64 = polish_x ? pass_grid<PASS_F64X, false, true>(P.W) : pass_grid<PASS_F64, false, true>(P.W);
    const bool use_x = prec == TC_F64X || (polish_x && prm->polish_steps > 0);
    const int64_t G_e = pass_grid<PASS_F64, true, false>(P.W);
    const int64_t G_d = pass_grid<PASS_DELTA, false, false>(P.W);
    const bool ls_on = lbfgs && prm->line_search > 0;
    const int64_t G_dm = pass_grid<PASS_DMIX, false, false>(P.W);
    // the mixed bulk pass: its persistent CTAs take equal ranges from a queue (mixed_ranges), so
    // units of uneven cost (tiles that turn near as subdomains spread, partial row blocks) stay
    // balanced over the SMs
    // instances: the float64 passes take each unordered pair once and their ranges from the queue
    int64_t rb_max = 0;
    for (const Prob& p : P.prob) rb_max = std::max<int64_t>(rb_max, p.n_rb);
    const bool sym = inst && rb_max * P.M * 24 <= kSymBytes;
    const int64_t G_sym = sym ? sym_ranges(P.W) : 0;
    const int64_t G_rng = prec == TC_MIXED ? mixed_ranges(P.W) : (sym && prec == TC_FP64 ? G_sym : G_bulk);
    const int64_t G_pol = sym && !polish_x ? G_sym : G_f64;
    const int64_t G_en = sym ? G_sym : G_e;
    int64_t slots = 1;
    for (int64_t G : {G_rng, G_pol, G_en, G_d, G_dm}) slots = std::max(slots, plan_slots(P.prob, 0, P.prob.size(), 0, P.W, G));
    // phases whose gradient passes leave many slots per row sum them over every SM before the update
    const bool pre_bulk = plan_slots(P.prob, 0, P.prob.size(), 0, P.W, G_rng) > kPreReduceSlots;
    const bool pre_polish = plan_slots(P.prob, 0, P.prob.size(), 0, P.W, G_pol) > kPreReduceSlots;
    // single-problem passes of the sequential accept: R1[k] ranges of one to two units, taken from
    // the queue by C1[k] persistent CTAs, so the cheap units of a partial last row block do not
    // leave SMs idle while others finish whole row blocks; with many slots per row, the rows'
    // partials are summed over every SM (k_sum_slots_e) before the one-CTA accept kernel
    int64_t slots1 = 1;
    std::vector<int64_t> R1(n_sub), C1(n_sub);
    if (!inst && prm->accept) {
        for (int32_t k = 0; k < n_sub; ++k) {
            const Prob& p = P.prob[k];
            int64_t Wk = (int64_t)p.n_rb * (p.n_t_snap + p.n_t_priv);
            R1[k] = std::max<int64_t>(1, sym_ranges(Wk));
            C1[k] = mixed_ctas(R1[k], std::min<int64_t>(G_d, R1[k]));
            slots1 = std::max(slots1, plan_slots(P.prob, k, k + 1, p.unit_off, Wk, R1[k]));
        }
    }
    const bool pre_accept = slots1 > kPreReduceSlots;
    const int64_t M = P.M;
    const int64_t taken_words = (n + 31) / 32;
    LargeSet large;
    // L-BFGS-B steps every problem on one CTA or cluster (launch_lbfgsb), whatever its size
    if (lbfgs && !boxed)
        for (int32_t k = 0; k < n_sub; ++k)
            if (P.prob[k].m > kLargeRows) large.ids.push_back(k);

    // more one-CTA L-BFGS problems than resident update CTAs: persistent CTAs take them largest
    // first from a queue, so the float64 work of the big problems spreads over the SMs
    std::vector<int32_t> upd_order;
    const int upd_ctas = kUpdPerSm * sm_count();
    if (lbfgs && !boxed && n_sub > upd_ctas) {
        for (int32_t k = 0; k < n_sub; ++k)
            if (P.prob[k].m <= kLargeRows) upd_order.push_back(k);
        std::stable_sort(upd_order.begin(), upd_order.end(),
                         [&](int32_t a_, int32_t b_) { return P.prob[a_].m > P.prob[b_].m; });
    }

    Carver c;
    fx3* snap3 = nullptr;
    int32_t* upd_order_d = nullptr;
    double2* col_g = nullptr;
    double* col_e = nullptr;
    double* acc_red = nullptr;
    auto layout = [&](Carver& cv, RelaxDev& d, Prob*& probd, int64_t*& wbd, float4*& snap_split, double*& part_e,
                      double2*& part_g, double*& part1) {
        probd = cv.take<Prob>(n_sub);
        wbd = cv.take<int64_t>(n_sub);
        d.gidx = cv.take<int32_t>(M);
        d.x = cv.take<double2>(M);
        d.xs = cv.take<float4>(M);
        d.x3 = use_x ? cv.take<fx3>(M) : nullptr;
        snap3 = cv.take<fx3>(use_x && !inst ? n : 0);
        d.g = cv.take<double2>(M);
        d.g_red = cv.take<double2>(pre_bulk || pre_polish ? M : 0);
        col_g = cv.take<double2>(sym ? (size_t)(rb_max * M) : 0);
        col_e = cv.take<double>(sym ? (size_t)(rb_max * M) : 0);
        d.xp = cv.take<double2>(M);
        d.gp = cv.take<double2>(M);
        d.z = cv.take<double2>(lbfgs ? M : 0);
        d.q = cv.take<double2>(lbfgs ? M : 0);
        d.Sh = cv.take<double2>(lbfgs ? (size_t)mem * M : 0);
        d.Yh = cv.take<double2>(lbfgs ? (size_t)mem * M : 0);
        d.bp = cv.take<double>(boxed ? M : 0);
        d.xc = cv.take<double2>(boxed ? M : 0);
        d.bsmall = cv.take<double>(boxed ? (size_t)n_sub * kBSmall : 0);
        d.any_active = cv.take<int>(1);
        d.rows4 = cv.take<d4>(M);
        d.rows8 = ls_on ? cv.take<f8>(M) : nullptr;
        d.xold = ls_on ? cv.take<double2>(M) : nullptr;
        d.ls_alpha = ls_on ? cv.take<double>(n_sub) : nullptr;
        d.ls_gd = ls_on ? cv.take<double>(n_sub) : nullptr;
        d.ls_active = ls_on ? cv.take<int>(n_sub) : nullptr;
        d.mask = cv.take<uint32_t>(mask_words);
        d.taken = cv.take<uint32_t>(taken_words);
        d.active = cv.take<int>(n_sub);
        d.ok = cv.take<int>(n_sub);
        d.steps = cv.take<int>(n_sub);
        d.hist = cv.take<int>(n_sub);
        d.head = cv.take<int>(n_sub);
        d.status = cv.take<int>(n_sub);
        d.rho = cv.take<double>((size_t)n_sub * kMaxMem);
        d.gram = cv.take<double>(lbfgs && !boxed ? (size_t)n_sub * kLbGram : 0);
        d.rms = cv.take<double>(n_sub);
        d.delta = cv.take<double>(n_sub);
        d.energy = cv.take<double>(n_sub);
        snap_split = cv.take<float4>(inst ? 0 : n);
        large.part = cv.take<double>(lbfgs ? (size_t)kLbPasses * kLargeBlocks * kLbVals : 0);
        large.sc = cv.take<LbCoef>(lbfgs ? large.ids.size() : 0);
        part_e = cv.take<double>(slots * M);
        part_g = cv.take<double2>(slots * M);
        part1 = cv.take<double>(slots1 * max_m);
        acc_red = cv.take<double>(pre_accept ? max_m : 0);
        upd_order_d = cv.take<int32_t>(upd_order.size());
    };
    RelaxDev d{};
    Prob* probd;
    int64_t* wbd;
    float4* snap_split;
    double *part_e, *part1;
    double2* part_g;
    layout(c, d, probd, wbd, snap_split, part_e, part_g, part1);
    void* ws = workspace(s, c.off, &err);
    if (!ws) return err;
    c.base = static_cast<char*>(ws);
    c.off = kCounterBytes;
    layout(c, d, probd, wbd, snap_split, part_e, part_g, part1);
    d.prob = probd;
    d.S = n_sub;
    d.M = M;
    d.wbeg = wbd;
    d.idx = idx;
    d.flags = flags;
    d.pos = reinterpret_cast<double2*>(pos);
    d.st = st;
    d.tu = prm->optimizer == TC_OPT_LBFGS_TU || boxed ? 1 : 0;
    d.boxed = boxed ? 1 : 0;
    if (!upd_order.empty()) {
        d.upd_order = upd_order_d;
        d.upd_n = (int)upd_order.size();
        d.upd_ctas = upd_ctas;
        d.upd_ctr = reinterpret_cast<unsigned*>(static_cast<char*>(ws) + kUpdCtrOff);
    }

    cudaError_t e = cudaSuccess;
    if (prof) cudaEventRecord(ev_a, s);
    e = cudaMemcpyAsync(probd, P.prob.data(), sizeof(Prob) * n_sub, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(wbd, wbeg.data(), 8 * (size_t)n_sub, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !upd_order.empty())
        e = cudaMemcpyAsync(upd_order_d, upd_order.data(), 4 * upd_order.size(), cudaMemcpyHostToDevice, s);
    // the queues' counters start every call at zero, whatever an earlier failed call left
    if (e == cudaSuccess && d.upd_ctr) e = cudaMemsetAsync(d.upd_ctr, 0, sizeof(unsigned), s);
    unsigned* pass_ctr = reinterpret_cast<unsigned*>(static_cast<char*>(ws) + kPassCtrOff);
    if (e == cudaSuccess) e = cudaMemsetAsync(pass_ctr, 0, sizeof(unsigned), s);
    // per-problem state: active = ok = 1, counters zero
    std::vector<int> ones(n_sub, 1);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d.active, ones.data(), 4 * (size_t)n_sub, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d.ok, ones.data(), 4 * (size_t)n_sub, cudaMemcpyHostToDevice, s);
    for (int* z : {d.steps, d.hist, d.head, d.status})
        if (e == cudaSuccess) e = cudaMemsetAsync(z, 0, 4 * (size_t)n_sub, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.rms, 0, 8 * (size_t)n_sub, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.delta, 0, 8 * (size_t)n_sub, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.energy, 0, 8 * (size_t)n_sub, s);
    if (e == cudaSuccess && mask_words) e = cudaMemsetAsync(d.mask, 0, 4 * (size_t)mask_words, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.taken, 0, 4 * (size_t)taken_words, s);
    if (e != cudaSuccess) return cuda_fail(e, "set-up");
    const int eb = (int)std::max<int64_t>(1, std::min<int64_t>((M + 255) / 256, 8L * sm_count()));
    if (M > 0) {
        k_rows_init<<<eb, 256, 0, s>>>(d, n, prm->radius, lbfgs ? 1 : 0);
        ++launches;
        if (!inst) {
            k_mask_build<<<eb, 256, 0, s>>>(d);
            ++launches;
        }
    }
    if (!inst && n > 0) {
        int nb = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8L * sm_count()));
        k_split_pos<<<nb, 256, 0, s>>>(reinterpret_cast<const double2*>(pos), n, snap_split, st);
        ++launches;
        if (use_x) {
            k_split3_pos<<<nb, 256, 0, s>>>(reinterpret_cast<const double2*>(pos), n, snap3);
            ++launches;
        }
    }
    if (prof) cudaEventRecord(ev_b, s);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "launch");
    // argument errors found on the device stop the call before any step
    {
        int hst = 0;
        if (cudaError_t e_ = cudaMemcpyAsync(&hst, st, 4, cudaMemcpyDeviceToHost, s); e_ != cudaSuccess)
            return cuda_fail(e_, "status read");
        if (cudaError_t e_ = cudaStreamSynchronize(s); e_ != cudaSuccess) return cuda_fail(e_, "set-up");
        if (hst != 0) {
            cudaMemsetAsync(st, 0, 4, s);
            cudaStreamSynchronize(s);
            return static_cast<tc_status>(hst);
        }
    }

    PassArgs a{};
    a.prob = probd;
    a.S = n_sub;
    a.W = P.W;
    a.M = M;
    a.mask = inst ? nullptr : d.mask;
    a.active = d.active;
    a.part_e = part_e;
    a.part_g = part_g;
    StepParams sp{prm->optimizer, mem, prm->step0, prm->alpha_min, prm->alpha_max, prm->maxstep, prm->gtol, prm->radius, 0};
    sp.line_search = ls_on ? prm->line_search : 0;
    sp.pre_reduce = pre_bulk ? 1 : 0;
    // energy-change passes of the line search: float32 difference form in the mixed phase,
    // float64 pair differences otherwise (rows: rows8 / rows4; snapshot as the relaxation's)
    LsArgs ls_mixed, ls_f64;
    ls_mixed.a = a;
    ls_mixed.a.rows = d.rows8;
    ls_mixed.a.snap = snap_split;
    ls_mixed.a.active = d.ls_active;
    ls_mixed.a.part_g = nullptr;
    ls_mixed.G = G_dm;
    ls_mixed.mixed = true;
    ls_f64.a = a;
    ls_f64.a.rows = d.rows4;
    ls_f64.a.snap = pos;
    ls_f64.a.active = d.ls_active;
    ls_f64.a.part_g = nullptr;
    ls_f64.G = G_d;
    // the float64 passes' arguments (symmetric and queued for instances), for up to ctas_max CTAs
    auto f64args = [&](int64_t ctas_max) {
        PassArgs x = a;
        x.rows = d.x;
        x.snap = pos;
        if (sym) {
            x.sym = 1;
            x.col_g = col_g;
            x.col_e = col_e;
            x.col_stride = M;
            x.ticket = pass_ctr;
            x.ctas = mixed_ctas(G_sym, ctas_max);
        }
        return x;
    };
    tc_status rs;
    if (prec == TC_MIXED) {
        PassArgs ab = a;
        ab.rows = d.xs;
        ab.snap = snap_split;
        ab.ticket = pass_ctr;
        ab.ctas = mixed_ctas(G_rng, G_bulk);
        rs = run_phase<PASS_MIXED>(d, ab, P, G_rng, sp, prm->n_steps, s, prof, launches, large, &ls_mixed);
    } else if (prec == TC_F64X) {
        a.rows = d.x3;
        a.snap = snap3;
        rs = run_phase<PASS_F64X>(d, a, P, G_bulk, sp, prm->n_steps, s, prof, launches, large, &ls_f64);
    } else {
        rs = run_phase<PASS_F64>(d, f64args(sym ? pass_grid<PASS_F64, false, true, true>(P.W) : G_bulk), P, G_rng, sp,
                                 prm->n_steps, s, prof, launches, large, &ls_f64);
    }
    if (rs != TC_OK) return rs;
    if (prm->polish_steps > 0) {
        // float64 polish: every problem steps again, L-BFGS history kept
        if (cudaError_t e_ = cudaMemcpyAsync(d.active, ones.data(), 4 * (size_t)n_sub, cudaMemcpyHostToDevice, s); e_ != cudaSuccess) return cuda_fail(e_, "cudaMemcpyAsync");
        StepParams sp2 = sp;
        sp2.gtol = prm->polish_gtol;
        sp2.pre_reduce = pre_polish ? 1 : 0;
        if (polish_x) {
            a.rows = d.x3;
            a.snap = snap3;
            rs = run_phase<PASS_F64X>(d, a, P, G_f64, sp2, prm->polish_steps, s, prof, launches, large, &ls_f64);
        } else {
            rs = run_phase<PASS_F64>(d, f64args(sym ? pass_grid<PASS_F64, false, true, true>(P.W) : G_f64), P, G_pol,
                                     sp2, prm->polish_steps, s, prof, launches, large, &ls_f64);
        }
        if (rs != TC_OK) return rs;
    }
    a.active = nullptr;
    if (prof) cudaEventRecord(ev_c, s);
    if (prm->want_energy) {
        // float64 E_sub of the relaxed rows against the entry configuration
        const PassArgs ae = f64args(sym ? pass_grid<PASS_F64, true, false, true>(P.W) : G_e);
        if ((e = launch_pass<PASS_F64, true, false>(ae, G_en, 0, 0, s)) != cudaSuccess) return cuda_fail(e, "launch");
        const SlotView v = pass_view(ae, P.W, G_en, M);
        k_problem_sums<<<n_sub, kUpd, 0, s>>>(d, part_e, v, d.energy, nullptr);
        launches += (P.W > 0 ? 1 : 0) + 1;
    }
    if (prm->accept) {
        k_rows4<<<eb, 256, 0, s>>>(d, d.x);
        ++launches;
        a.rows = d.rows4;
        a.snap = pos;
        if (inst) {
            if ((e = launch_pass<PASS_DELTA, false, false>(a, G_d, 0, 0, s)) != cudaSuccess) return cuda_fail(e, "launch");
            SlotView v{P.W, G_d, 0, M, 0};
            k_problem_sums<<<n_sub, kUpd, 0, s>>>(d, part_e, v, d.delta, nullptr);
            k_write_back<<<eb, 256, 0, s>>>(d, 1);
            launches += (P.W > 0 ? 1 : 0) + 2;
        } else {
            a.part_e = part1;
            a.active = d.ok;
            for (int32_t k = 0; k < n_sub; ++k) {
                const Prob& p = P.prob[k];
                PassArgs ak = a;
                ak.W = (int64_t)p.n_rb * (p.n_t_snap + p.n_t_priv);
                ak.M = std::max<int64_t>(p.m, 1);
                ak.ticket = pass_ctr;
                ak.ctas = C1[k];
                if ((e = launch_pass<PASS_DELTA, false, false>(ak, R1[k], p.unit_off, p.row_base, s)) != cudaSuccess)
                    return cuda_fail(e, "accept pass launch");
                SlotView v{ak.W, R1[k], p.unit_off, ak.M, p.row_base};
                if (pre_accept && p.m > 0) {
                    k_sum_slots_e<<<(unsigned)((p.m + 255) / 256), 256, 0, s>>>(d, k, part1, v, acc_red);
                    v.rede = acc_red;
                    ++launches;
                }
                k_accept_apply<<<1, kUpd, 0, s>>>(d, k, part1, v);
                launches += (ak.W > 0 ? 1 : 0) + 1;
            }
        }
    } else if (inst) {
        k_write_back<<<eb, 256, 0, s>>>(d, 0);
        ++launches;
    }
    k_results<<<(n_sub + 127) / 128, 128, 0, s>>>(d, out, inst ? 1 : 0, prm->accept ? 1 : 0, prm->want_energy ? 1 : 0);
    ++launches;
    if (prof) cudaEventRecord(ev_d, s);
    if (cudaError_t e_ = cudaGetLastError(); e_ != cudaSuccess) return cuda_fail(e_, "cudaGetLastError");
    e = cudaStreamSynchronize(s);
    if (prof && e == cudaSuccess) {
        g_last_profile.setup_ms = elapsed(ev_a, ev_b);
        g_last_profile.accept_ms = elapsed(ev_c, ev_d);
    }
    g_last_profile.launches = launches;
    int64_t pairs = 0;
    for (const Prob& p : P.prob) {
        // a row meets every other charge of its world once: m (world - 1) in
        // subdomain mode, m (m - 1) for an instance
        int64_t others = inst ? (int64_t)p.m - 1 : (p.snap_e - p.snap_b) - 1;
        pairs += (int64_t)p.m * std::max<int64_t>(others, 0);
    }
    g_last_profile.pass_pairs = pairs;
    return cuda_status(e, "relaxation (accept / write-back / results)");
}

// tc_subdomain_delta_energy: every subdomain against pos, in one pass.
// Energy change of every subdomain against pos: float64 pair differences
// (mixed = false) or the float32 difference form with its error bound.
static tc_status delta_all(const double* pos, int64_t n, const int32_t* idx, const int64_t* offsets, int32_t n_sub,
                           const double* new_active, double* delta, bool mixed, double* bound, cudaStream_t s)
{
    if (n < 0 || n_sub < 0 || (n > 0 && !pos) || (n_sub > 0 && (!offsets || !delta)) ||
        (reinterpret_cast<uintptr_t>(pos) & 15) || (reinterpret_cast<uintptr_t>(new_active) & 15) ||
        (reinterpret_cast<uintptr_t>(delta) & 7) || (reinterpret_cast<uintptr_t>(bound) & 7))
        return TC_ERR_INVALID_ARG;
    if (n_sub == 0) return TC_OK;
    if (n > INT32_MAX) return TC_ERR_INVALID_ARG;
    tc_status err = TC_OK;
    int* st = device_status(&err);
    if (!st) return err;
    std::vector<int64_t> off(n_sub + 1);
    if (cudaError_t e_ = cudaMemcpyAsync(off.data(), offsets, 8 * (size_t)(n_sub + 1), cudaMemcpyDeviceToHost, s);
        e_ != cudaSuccess)
        return cuda_fail(e_, "offsets read");
    if (cudaError_t e_ = cudaStreamSynchronize(s); e_ != cudaSuccess) return cuda_fail(e_, "offsets read");
    Plan P;
    P.prob.resize(n_sub);
    int64_t mask_words = 0;
    if (off[0] != 0) return TC_ERR_INVALID_ARG;
    for (int32_t k = 0; k < n_sub; ++k) {
        if (off[k + 1] < off[k] || off[k + 1] - off[k] > n) return TC_ERR_INVALID_ARG;
        Prob& p = P.prob[k];
        p.row_base = off[k];
        p.m = (int32_t)(off[k + 1] - off[k]);
        p.snap_b = 0;
        p.snap_e = n;
        p.mask_off = mask_words;
        mask_words += (n + 31) / 32;
    }
    P.M = off[n_sub];
    if (P.M > 0 && (!idx || !new_active)) return TC_ERR_INVALID_ARG;
    plan_units(P);
    const int64_t G = mixed ? pass_grid<PASS_DMIX, false, false>(P.W) : pass_grid<PASS_DELTA, false, false>(P.W);
    // float64: the persistent CTAs take ranges of a few units from the queue (sym_ranges), so the
    // cheap units of partial last row blocks leave no SM idle while others finish whole blocks
    const int64_t R = mixed ? G : sym_ranges(P.W);
    const int64_t slots = plan_slots(P.prob, 0, P.prob.size(), 0, P.W, R);
    const int64_t M = P.M;
    Carver c;
    f8* rows8 = nullptr;
    float4* snap_split = nullptr;
    double2* part_b = nullptr;
    auto layout = [&](Carver& cv, RelaxDev& d, Prob*& probd, double*& part_e) {
        probd = cv.take<Prob>(n_sub);
        d.gidx = cv.take<int32_t>(M);
        d.rows4 = cv.take<d4>(mixed ? 0 : M);
        rows8 = cv.take<f8>(mixed ? M : 0);
        snap_split = cv.take<float4>(mixed ? n : 0);
        d.mask = cv.take<uint32_t>(mask_words);
        part_e = cv.take<double>(slots * std::max<int64_t>(M, 1));
        part_b = cv.take<double2>(mixed ? slots * std::max<int64_t>(M, 1) : 0);
    };
    RelaxDev d{};
    Prob* probd;
    double* part_e;
    layout(c, d, probd, part_e);
    void* ws = workspace(s, c.off, &err);
    if (!ws) return err;
    c.base = static_cast<char*>(ws);
    c.off = kCounterBytes;
    layout(c, d, probd, part_e);
    d.prob = probd;
    d.S = n_sub;
    d.M = M;
    d.idx = idx;
    d.pos = const_cast<double2*>(reinterpret_cast<const double2*>(pos));
    d.st = st;
    cudaError_t e = cudaMemcpyAsync(probd, P.prob.data(), sizeof(Prob) * n_sub, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.mask, 0, 4 * (size_t)mask_words, s);
    if (e != cudaSuccess) return cuda_fail(e, "set-up");
    const int eb = (int)std::max<int64_t>(1, std::min<int64_t>((M + 255) / 256, 8L * sm_count()));
    if (M > 0) {
        d.x = nullptr;
        d.xs = nullptr;
        k_rows_init<<<eb, 256, 0, s>>>(d, n, 1.0, 0);
        k_mask_build<<<eb, 256, 0, s>>>(d);
        if (mixed) {
            const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8L * sm_count()));
            k_split_pos<<<nb, 256, 0, s>>>(reinterpret_cast<const double2*>(pos), n, snap_split, st);
            k_rows8<<<eb, 256, 0, s>>>(d, reinterpret_cast<const double2*>(new_active), rows8);
        } else {
            k_rows4<<<eb, 256, 0, s>>>(d, reinterpret_cast<const double2*>(new_active));
        }
    }
    PassArgs a{};
    a.prob = probd;
    a.S = n_sub;
    a.W = P.W;
    a.M = std::max<int64_t>(M, 1);
    a.rows = mixed ? static_cast<const void*>(rows8) : static_cast<const void*>(d.rows4);
    a.snap = mixed ? static_cast<const void*>(snap_split) : static_cast<const void*>(pos);
    a.mask = d.mask;
    a.active = nullptr;
    a.part_e = part_e;
    a.part_g = part_b;
    SlotView v{P.W, R, 0, a.M, 0};
    if (mixed) {
        if ((e = launch_pass<PASS_DMIX, false, false>(a, G, 0, 0, s)) != cudaSuccess) return cuda_fail(e, "launch");
        k_dmix_sums<<<n_sub, kUpd, 0, s>>>(d, part_e, part_b, v, delta, bound);
    } else {
        a.ticket = reinterpret_cast<unsigned*>(static_cast<char*>(ws) + kPassCtrOff);
        a.ctas = mixed_ctas(R, G);
        if ((e = cudaMemsetAsync(a.ticket, 0, sizeof(unsigned), s)) != cudaSuccess) return cuda_fail(e, "set-up");
        if ((e = launch_pass<PASS_DELTA, false, false>(a, R, 0, 0, s)) != cudaSuccess) return cuda_fail(e, "launch");
        k_problem_sums<<<n_sub, kUpd, 0, s>>>(d, part_e, v, delta, nullptr);
    }
    return cuda_status(cudaGetLastError());
}

// ------------------------------------------------------ subdomain gradient ---

// Rows of the subdomain gradient at caller-given active positions: the float64
// copy and the split the pass of that precision reads.
__global__ void k_rows_act(RelaxDev d, const double2* __restrict__ act)
{
    for (int64_t rr = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; rr < d.M; rr += (int64_t)gridDim.x * blockDim.x) {
        const double2 x = act[rr];
        if (!isfinite(x.x) || !isfinite(x.y)) set_status(d.st, ST_NONFINITE);
        else if (!inside(x.x, x.y)) set_status(d.st, ST_OUTSIDE);
        if (d.x) d.x[rr] = x;
        if (d.xs) d.xs[rr] = split4(x.x, x.y);
        if (d.x3) d.x3[rr] = split3(x.x, x.y);
    }
}

// Per row: the slots of the pass added in order (the reduction every update
// kernel starts with), written out as dE_sub/da and e_k.
__global__ void k_rows_out(RelaxDev d, const double* __restrict__ part_e, const double2* __restrict__ part_g,
                           SlotView v, double2* __restrict__ grad, double* __restrict__ local_e)
{
    for (int64_t rr = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; rr < d.M; rr += (int64_t)gridDim.x * blockDim.x) {
        const int s = find_row_prob(d.prob, d.S, rr);
        const Prob p = d.prob[s];
        const int64_t rl = rr - p.row_base;
        const double2 g = sum_g(p, rl, part_g, v);
        const double e = sum_e(p, rl, part_e, v);
        if (!isfinite(g.x) || !isfinite(g.y) || !isfinite(e)) set_status(d.st, ST_NONFINITE);
        grad[rr] = g;
        if (local_e) local_e[rr] = e;
    }
}

template <int KIND>
static cudaError_t subgrad_pass(const PassArgs& a, int64_t G, cudaStream_t s)
{
    return launch_pass<KIND, true, true>(a, G, 0, 0, s);
}

// tc_subdomain_grad: the relaxation's pair pass, once, at given active positions.
static tc_status subdomain_grad(const double* pos, int64_t n, const int32_t* idx, const int64_t* offsets,
                                int32_t n_sub, const double* act, int prec, double* grad, double* local_e,
                                double* e_sub, cudaStream_t s)
{
    if (prec != TC_FP64 && prec != TC_MIXED && prec != TC_F64X) return TC_ERR_INVALID_ARG;
    if (n < 0 || n_sub < 0 || (n > 0 && !pos) || (n_sub > 0 && !offsets) || (reinterpret_cast<uintptr_t>(pos) & 15) ||
        (reinterpret_cast<uintptr_t>(act) & 15) || (reinterpret_cast<uintptr_t>(grad) & 15) ||
        (reinterpret_cast<uintptr_t>(local_e) & 7) || (reinterpret_cast<uintptr_t>(e_sub) & 7))
        return TC_ERR_INVALID_ARG;
    if (n_sub == 0) return TC_OK;
    if (n > INT32_MAX) return TC_ERR_INVALID_ARG;
    tc_status err = TC_OK;
    int* st = device_status(&err);
    if (!st) return err;
    std::vector<int64_t> off(n_sub + 1);
    if (cudaError_t e_ = cudaMemcpyAsync(off.data(), offsets, 8 * (size_t)(n_sub + 1), cudaMemcpyDeviceToHost, s);
        e_ != cudaSuccess)
        return cuda_fail(e_, "offsets read");
    if (cudaError_t e_ = cudaStreamSynchronize(s); e_ != cudaSuccess) return cuda_fail(e_, "offsets read");
    Plan P;
    P.prob.resize(n_sub);
    int64_t mask_words = 0;
    if (off[0] != 0) return TC_ERR_INVALID_ARG;
    for (int32_t k = 0; k < n_sub; ++k) {
        if (off[k + 1] < off[k] || off[k + 1] - off[k] > n) return TC_ERR_INVALID_ARG;
        Prob& p = P.prob[k];
        p.row_base = off[k];
        p.m = (int32_t)(off[k + 1] - off[k]);
        p.snap_b = 0;
        p.snap_e = n;
        p.mask_off = mask_words;
        mask_words += (n + 31) / 32;
    }
    P.M = off[n_sub];
    if (P.M > 0 && (!idx || !grad)) return TC_ERR_INVALID_ARG;
    plan_units(P);
    const int64_t G = prec == TC_MIXED  ? pass_grid<PASS_MIXED, true, true>(P.W)
                      : prec == TC_F64X ? pass_grid<PASS_F64X, true, true>(P.W)
                                        : pass_grid<PASS_F64, true, true>(P.W);
    const int64_t slots = plan_slots(P.prob, 0, P.prob.size(), 0, P.W, G);
    const int64_t M = P.M;
    const int64_t Mp = std::max<int64_t>(M, 1);
    Carver c;
    float4* snap_split = nullptr;
    fx3* snap3 = nullptr;
    auto layout = [&](Carver& cv, RelaxDev& d, Prob*& probd, double*& part_e, double2*& part_g) {
        probd = cv.take<Prob>(n_sub);
        d.gidx = cv.take<int32_t>(M);
        d.x = cv.take<double2>(M);
        d.xs = cv.take<float4>(prec == TC_MIXED ? M : 0);
        d.x3 = cv.take<fx3>(prec == TC_F64X ? M : 0);
        snap_split = cv.take<float4>(prec == TC_MIXED ? n : 0);
        snap3 = cv.take<fx3>(prec == TC_F64X ? n : 0);
        d.mask = cv.take<uint32_t>(mask_words);
        part_e = cv.take<double>(slots * Mp);
        part_g = cv.take<double2>(slots * Mp);
    };
    RelaxDev d{};
    Prob* probd;
    double* part_e;
    double2* part_g;
    layout(c, d, probd, part_e, part_g);
    void* ws = workspace(s, c.off, &err);
    if (!ws) return err;
    c.base = static_cast<char*>(ws);
    c.off = kCounterBytes;
    layout(c, d, probd, part_e, part_g);
    if (prec != TC_MIXED) d.xs = nullptr;
    if (prec != TC_F64X) d.x3 = nullptr;
    d.prob = probd;
    d.S = n_sub;
    d.M = M;
    d.idx = idx;
    d.pos = const_cast<double2*>(reinterpret_cast<const double2*>(pos));
    d.st = st;
    cudaError_t e = cudaMemcpyAsync(probd, P.prob.data(), sizeof(Prob) * n_sub, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.mask, 0, 4 * (size_t)mask_words, s);
    if (e != cudaSuccess) return cuda_fail(e, "set-up");
    const int eb = (int)std::max<int64_t>(1, std::min<int64_t>((M + 255) / 256, 8L * sm_count()));
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8L * sm_count()));
    if (M > 0) {
        k_rows_init<<<eb, 256, 0, s>>>(d, n, 1.0, 0);
        k_mask_build<<<eb, 256, 0, s>>>(d);
        if (act) k_rows_act<<<eb, 256, 0, s>>>(d, reinterpret_cast<const double2*>(act));
    }
    if (prec == TC_MIXED) k_split_pos<<<nb, 256, 0, s>>>(reinterpret_cast<const double2*>(pos), n, snap_split, st);
    if (prec == TC_F64X) k_split3_pos<<<nb, 256, 0, s>>>(reinterpret_cast<const double2*>(pos), n, snap3);
    PassArgs a{};
    a.prob = probd;
    a.S = n_sub;
    a.W = P.W;
    a.M = Mp;
    a.mask = d.mask;
    a.active = nullptr;
    a.part_e = part_e;
    a.part_g = part_g;
    if (prec == TC_MIXED) {
        a.rows = d.xs;
        a.snap = snap_split;
        e = subgrad_pass<PASS_MIXED>(a, G, s);
    } else if (prec == TC_F64X) {
        a.rows = d.x3;
        a.snap = snap3;
        e = subgrad_pass<PASS_F64X>(a, G, s);
    } else {
        a.rows = d.x;
        a.snap = pos;
        e = subgrad_pass<PASS_F64>(a, G, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "launch");
    SlotView v{P.W, G, 0, Mp, 0};
    if (M > 0) k_rows_out<<<eb, 256, 0, s>>>(d, part_e, part_g, v, reinterpret_cast<double2*>(grad), local_e);
    if (e_sub) k_problem_sums<<<n_sub, kUpd, 0, s>>>(d, part_e, v, e_sub, nullptr);
    return cuda_status(cudaGetLastError());
}

}  // namespace tc

extern "C" {

tc_status tc_subdomain_grad(const double* pos, int64_t n, const int32_t* idx, const int64_t* offsets, int32_t n_sub,
                            const double* act, tc_precision prec, double* grad, double* local_e, double* e_sub,
                            tc_stream stream)
{
    tc::NvtxRange nvtx_range("tc_subdomain_grad");
    return tc::subdomain_grad(pos, n, idx, offsets, n_sub, act, prec, grad, local_e, e_sub,
                              reinterpret_cast<cudaStream_t>(stream));
}

tc_status tc_relax_subdomains(double* pos, int64_t n, const int32_t* idx, const int64_t* offsets, int32_t n_sub,
                              const int64_t* world, const uint8_t* flags, const tc_relax_params* prm,
                              tc_subdomain_result* out, tc_stream stream)
{
    tc::NvtxRange nvtx_range("tc_relax_subdomains");
    return tc::relax(pos, n, idx, offsets, n_sub, world, flags, prm, out, reinterpret_cast<cudaStream_t>(stream));
}

tc_status tc_relax_last_profile(tc_relax_profile* out)
{
    if (!out) return TC_ERR_INVALID_ARG;
    *out = tc::g_last_profile;
    return TC_OK;
}

tc_status tc_subdomain_delta_energy(const double* pos, int64_t n, const int32_t* idx, const int64_t* offsets,
                                    int32_t n_sub, const double* new_active, double* delta, tc_stream stream)
{
    tc::NvtxRange nvtx_range("tc_subdomain_delta_energy");
    return tc::delta_all(pos, n, idx, offsets, n_sub, new_active, delta, false, nullptr,
                         reinterpret_cast<cudaStream_t>(stream));
}

tc_status tc_subdomain_delta_energy_mixed(const double* pos, int64_t n, const int32_t* idx, const int64_t* offsets,
                                          int32_t n_sub, const double* new_active, double* delta, double* bound,
                                          tc_stream stream)
{
    tc::NvtxRange nvtx_range("tc_subdomain_delta_energy_mixed");
    return tc::delta_all(pos, n, idx, offsets, n_sub, new_active, delta, true, bound,
                         reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
