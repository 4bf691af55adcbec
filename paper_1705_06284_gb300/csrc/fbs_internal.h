// Internal declarations shared by the library's translation units.
// Not part of the public ABI (that is include/fbs.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "fbs.h"

namespace fbs {

// ---------------------------------------------------------------- errors
void set_error(const std::string &msg);
struct Failure {
    fbs_status status;
    std::string msg;
};
// Throws Failure on CUDA error (caught at the ABI boundary).
void check_cuda(cudaError_t e, const char *what);
#define FBS_CUDA(call) ::fbs::check_cuda((call), #call)

// ---------------------------------------------------------------- FFT plan
// Radix factorisation of a length-n transform (n = 2^a 3^b <= 512).
struct FftFactors {
    int n;
    int nst;
    int r[12];
};
FftFactors make_factors(int n);

// Per-bin geometry of the pruned inverse transform.
//   Rb    : largest |m_j| a mode of the bin can have (clamped to N/2).
//   Db    : bin box extent along x and y (2Rb+1, or N when it would exceed N).
//   Dzb   : bin box extent along z (Rb+1, or N/2+1).
//   A_off : offset (complex elements) of the bin's x-stage output A_b[x][jy][jz].
//   G_off : offset (complex elements) of the bin's y-stage output per slab.
//   box_off: offset (complex elements) of the spectrum box the bin reads (a
//            field's own box in batched evaluations; 0 otherwise).
struct BinGeom {
    int Rb, Db, Dzb, empty;
    long long thr_lo, thr_hi;
    long long A_off, G_off;
    long long box_off;
};

// Device-side description of the spectrum box (forward output):
//   Box[jx][jy][jz], jx,jy in [0, D), jz in [0, Dz), complex64.
struct BoxGeom {
    int N, R, D, Dz;
};

// Index <-> frequency for an axis of extent D holding m in [-R, R] (D = 2R+1)
// or the whole FFT axis (D == N).
__host__ __device__ inline int box_freq(int j, int D, int N) {
    if (D == N) return j < N / 2 ? j : j - N;
    return j <= D / 2 ? j : j - D;
}
__host__ __device__ inline int box_index(int m, int D) {
    return m >= 0 ? m : m + D;
}

// ---------------------------------------------------------------- contraction tasks
// Pair-grouped work list (host + device copies).  For bispectra an outer
// pair (b, c) carries inner items a (single bins); for trispectra an outer
// pair (c, d) carries inner pairs (a, b).  item_out is the output index.
struct TaskList {
    int npairs = 0, nitems = 0;
    std::vector<int> pb, pc, pstart;        // outer pair bins, CSR start (npairs+1)
    std::vector<int> ia, ib, iout;          // inner item bins (ib = -1 for triplets), output index
};

// ---------------------------------------------------------------- timing
enum KernelClass {
    KC_FWD_Z = 0,
    KC_FWD_Y,
    KC_FWD_X,
    KC_INV_X,
    KC_INV_Y,
    KC_INV_Z,
    KC_CONTRACT,
    KC_CONTRACT_TC,
    KC_QUAD,
    KC_QUAD_TC,
    KC_REDUCE,
    KC_COUNT,
    KC_NUM
};

struct Plan;

// ---------------------------------------------------------------- kernels (launch wrappers)
// fft.cu
void upload_forward_twiddles(Plan &root);
void upload_eval_twiddles(Plan &level);
// Forward transforms of one field (d_field) or of nf fields (d_fields, a
// device array of nf pointers) into nf consecutive zbuf / ybuf / box blocks.
void launch_forward(Plan &p, const float *d_field, const float *const *d_fields, int nf, float2 *zbuf,
                    float2 *ybuf, float2 *box);
void launch_forward_grid(Plan &p, int N, const BoxGeom &bx, const FftFactors &fN, const float2 *tw,
                         const float *d_field, const float *const *d_fields, int nf, float2 *zbuf, float2 *ybuf,
                         float2 *box);
void launch_inverse_x(Plan &p, bool indicator_fp64);
void launch_inverse_x_geom(Plan &p, const BinGeom *geom, int nb, int nvb);
void launch_inverse_yz_slab(Plan &p, int x0, int nx, float *islab);
void launch_inverse_yz_slab_geom(Plan &p, int x0, int nx, float *islab, const BinGeom *geom, int nb, int nvb,
                                 double *sq);
int zstage_row_groups(int N);
// FP64 count fields N_b on the octant (wtab: weights w(|m|^2) instead of 1).
void launch_count_fields_fp64_impl(Plan &p, double *noct, int bin0, int nb, double2 *A64,
                                   double2 *G64, const BinGeom *d_geom_grp, const double *wtab = nullptr);
// quad_counts.cu: exact ordered quadruple counts of the items (4 bins each,
// rows of the FP64 octant count fields noct) on the plan's grid.
struct U128 {
    uint64_t lo = 0, hi = 0;
};
// With dthr (thresholds on |q|^2 of nd diagonal shells) also the counts split
// by the shell of the diagonal q = m1 + m2: dout[item * nd + D].
void exact_quad_counts(Plan &p, const double *noct, const std::vector<int> &items, std::vector<U128> &out,
                       const std::vector<long long> *dthr = nullptr, std::vector<U128> *dout = nullptr);
// diagonal.cu (diagonal-resolved trispectrum)
void launch_field_product(Plan &p, const float *a, const float *b, float *out, long long n);
void launch_diag_gram(Plan &p, const float2 *F0, const float2 *F1, const long long *d_offs, int nq, const int *d_idx,
                      const float *d_w, const int *d_dstart, int nd, const int *d_qout, double scale, double *out);
void launch_diag_normalise(Plan &p, const double *num, const double *cnt, long long n, double cT, double *TD);
// contract.cu (FP64 count sums)
void launch_count_contraction(Plan &p, const double *noct, int nb_in_group, int bin0,
                              const int *d_items, int nitems, int arity, double *d_sums);
// contract.cu
// nf > 1: a batch of nf fields, field f's bins at rows f*nbins.. of islab and
// its partial rows at part_batch + f*part_blocks*items (nullptr: the plan's).
void launch_contract_fp32(Plan &p, const float *islab, long long npts, long long slab_stride,
                          bool quads, int nf = 1, double *part_batch = nullptr);
void launch_contract_tc(Plan &p, const float *islab, long long npts, long long slab_stride, bool quads,
                        int nf = 1, double *part_batch = nullptr);
bool tc_quads_usable(Plan &p);
// Triplets and quadruplets of a trispectrum plan in one tensor-core pass.
bool tc_fused_usable(Plan &p);
void launch_contract_tc_fused(Plan &p, const float *islab, long long npts, long long slab_stride);
void launch_level_reduce(Plan &level, bool quads);
void launch_level_reduce_batch(Plan &level, bool quads, int nf, const double *tpart, const double *sq,
                               double *tnum, double *sumsq);
void launch_normalise(Plan &root, bool quads);
void launch_normalise_batch(Plan &root, bool quads, int nf, const double *tnum, const double *sumsq, double *B,
                            double *P);
// Connected trispectrum of the last evaluation into d_Tc[nquad] (root).
void launch_connected(Plan &root, double *d_Tc);
std::vector<int> fast_grids();  // grids with compile-time-radix kernels for every inverse stage
void zero_partials(Plan &p, bool quads);
std::vector<int> item_groups(const TaskList &t, int cap);
int contract_blocks();

// ---------------------------------------------------------------- plan
// A plan is a root plus one or more evaluation levels.  The root owns the
// forward transform of the field, the spectrum box, the global tables (bins,
// closed triplets and quadruplets in output order, counts) and the outputs.
// A level (also a Plan, with root_ set) evaluates a subset of the bins on its
// own grid M and contracts the items assigned to it: every item's product of
// shell fields is a trigonometric polynomial of degree <= the sum of its
// bins' largest components R, so its sum is exact on any M above that sum.
// Local bin b of a level is global bin gbin[b]; local triplet t is global
// output gtrip[t] (quadruplets: gquad).  Levels allocate through the root and
// time their launches through it; they share the root's scratch buffers for
// the per-slab stages, since they run one after another on the root's stream.
struct Plan {
    Plan *root_ = nullptr;        // null for the root
    std::vector<Plan *> levels;   // root only
    std::vector<int> gbin, gtrip, gquad;   // level only: local -> global maps
    std::vector<int> pbin;        // level only: global bin of local bin b if its P is taken here, else -1
    int *d_gtrip = nullptr, *d_gquad = nullptr, *d_pbin = nullptr;
    int *d_errbuf = nullptr;      // root only: [0] this evaluation's wait-timeout code, [1] sticky copy
    // root only, connected trispectrum: per-bin geometry on the input grid (for
    // the shell moments of the spectrum box), unpaired quadruple counts,
    // the quadruplet table, moment partials [nbins][16][3], output staging
    std::vector<long long> selfconj;  // self-conjugate modes of each bin
    std::vector<double> nconn;
    double *d_nconn = nullptr, *d_mom_part = nullptr, *d_Tc = nullptr;
    int *d_quadtab = nullptr;
    Plan &root() { return root_ ? *root_ : *this; }
    int N = 0;
    double L = 0;
    int nbins = 0;
    int precision = 0;
    unsigned flags = 0;
    int tc_wide = 0;             // FBS_OPT_TC_WIDE
    int tc_roles = 0;            // FBS_OPT_TC_ROLES: 0 auto, 1 = 16 A warps, 2 = 8 A + 8 B warps
    int tc_chunk = 0;            // FBS_OPT_TC_CHUNK: 0 auto, 1 = 64-point chunks, 2 = 128 where they fit
    int tc_pairs = 0;            // FBS_OPT_TC_PAIRS: 0 greedy pair cover, 1 = pairs (b, c)
    int tc_merge = 0;            // FBS_OPT_TC_MERGE: 0 hi and lo rows of B in one MMA where it fits, 1 = never
    int tc_bstages = 0;          // FBS_OPT_TC_BSTAGES: 0 auto, 2..4 operand-B stages where they fit
    int tc_bfroma = 0;           // FBS_OPT_TC_BFROMA: 0 inner pair rows from operand A where it applies, 1 = never
    int tc_stack = 0;            // FBS_OPT_TC_STACK: 0 A's hi and lo stacked on M where it applies, 1 = never
    long long tc_wait_limit = 0; // FBS_OPT_TC_WAIT_LIMIT: hand-off wait limit in cycles (0 = default)
    cudaStream_t stream = nullptr;
    double create_ms = 0;
    double count_margin = 0;  // largest |sum N..N / N_pix - nearest integer| of the rounded counts

    std::vector<long long> thr;  // nbins+1
    std::vector<long long> shell;
    std::vector<BinGeom> geom;
    BoxGeom box{};               // forward spectrum box (transform length N)
    FftFactors fN{};
    int M = 0;                   // evaluation grid of the shell fields (M <= N)
    BoxGeom boxM{};              // the box seen by the inverse stages (transform length M)
    FftFactors fM{};
    float2 *d_twM = nullptr;     // e^{-2 pi i k/M}, k < M (FP32)

    std::vector<int32_t> trip;   // 3*ntrip
    std::vector<int64_t> ntri;
    std::vector<int32_t> quad;   // 4*nquad
    std::vector<double> nquad;   // FP64 ordered quadruple counts (the nearest double of nquad128)
    std::vector<U128> nquad128;  // exact ordered quadruple counts (root plan, output order)
    TaskList ttask, qtask;
    std::vector<int> tgrp, qgrp;  // item groups of the FP32 contraction (outer-pair ranges)
    int *d_tgrp = nullptr, *d_qgrp = nullptr;

    long long A_elems = 0;       // complex elements of the x-stage output (all bins)
    long long G_plane = 0;       // complex elements of the y-stage output per plane (all bins)
    int slab = 0;                // x planes per slab
    int nslabs = 0;
    int slab_planned = 0;        // planes per slab the buffers were sized for

    // device memory
    std::vector<void *> allocs;
    long long dev_bytes = 0;
    // timeout reporting: the normalisation copies the device's sticky flag
    // into h_err (pinned) at the end of every tensor-core evaluation and
    // records ev_err, so later calls can see a timeout without waiting
    int *h_err = nullptr;
    cudaEvent_t ev_err = nullptr;
    bool err_recorded = false;
    float *d_field = nullptr;    // staging for host fields
    cudaStream_t copy_stream = nullptr;   // host-field copies (overlap work queued on `stream`)
    cudaEvent_t ev_field_ready = nullptr; // staged copy landed (the plan's stream waits on it)
    cudaEvent_t ev_field_free = nullptr;  // the forward transform is done with the staging buffer
    bool field_free_recorded = false;
    float2 *d_zbuf = nullptr;    // forward scratch [N][N][Dz]
    float2 *d_ybuf = nullptr;    // forward scratch [N][D][Dz]
    float2 *d_box = nullptr;     // spectrum box [D][D][Dz]
    float2 *d_A = nullptr;       // inverse x-stage output
    float2 *d_G = nullptr;       // inverse y-stage output (one slab)
    float *d_I = nullptr;        // shell fields (one slab) [bin][plane][y][z]
    BinGeom *d_geom = nullptr;
    float2 *d_tw = nullptr;      // e^{-2 pi i k/N}, k < N (FP32)
    double2 *d_tw64 = nullptr;   // e^{-2 pi i k/M}, k < M, in FP64 (count fields)
    // task lists on device
    int *d_tpb = nullptr, *d_tpc = nullptr, *d_tps = nullptr, *d_tia = nullptr, *d_tout = nullptr;
    int *d_qpb = nullptr, *d_qpc = nullptr, *d_qps = nullptr, *d_qia = nullptr, *d_qib = nullptr,
        *d_qout = nullptr;
    // accumulators
    int part_blocks = 0;          // number of FP64 partial rows
    double *d_tpart = nullptr;    // [part_blocks][ntrip]
    double *d_qpart = nullptr;    // [part_blocks][nquad]
    double *d_fpart = nullptr;    // [part_blocks][ntrip + nquad] of the fused tensor-core pass
    bool fused_active = false;    // this evaluation uses the fused pass
    double *d_sumsq = nullptr;    // [nbins]
    double *d_sumsq_part = nullptr;  // [nbins][N][z-stage row groups]
    double *d_tnum = nullptr;     // [ntrip]
    double *d_qnum = nullptr;     // [nquad]
    double *d_B = nullptr, *d_P = nullptr, *d_T = nullptr;  // staging for host outputs
    int64_t *d_ntri = nullptr;
    double *d_nquad = nullptr;
    long long *d_shell = nullptr;
    // tensor-core path
    void *tc = nullptr;           // opaque state of contract_tc.cu
    void *batch = nullptr;        // root only: buffers of batched evaluations (plan.cpp)
    void *diag = nullptr;         // root only: diagonal-resolved trispectrum tables (plan.cpp)
    // root only: evaluate the spectrum box of another plan (fbs_plan_follow);
    // the plan's own box and its geometry are kept to detach
    const Plan *leader = nullptr;
    float2 *own_box = nullptr;
    BoxGeom own_boxgeom{};

    // timing
    std::vector<cudaEvent_t> evs;  // 2 per pending launch, created once and reused
    double kt_ms[KC_NUM] = {};
    long long kt_n[KC_NUM] = {};
    std::vector<std::pair<int, int>> pending;  // (class, event pair index)

    void *dalloc(size_t bytes);
    void tic(int cls, int &slot);
    void toc(int slot);
    void flush_times();
};

// Bracket a launch with timing events when FBS_FLAG_TIMING is set.
struct KTimer {
    Plan &p;
    int slot = -1;
    KTimer(Plan &pl, int cls) : p(pl) { p.tic(cls, slot); }
    ~KTimer() { p.toc(slot); }
};

void free_tc_state(Plan &p);
int *tc_error_flag(Plan &p);   // device flag set by a timed-out tensor-core wait (or nullptr)
void tc_job_info(Plan &p, int which, int32_t *out);  // job shape diagnostics (fbs_plan_tc_info)
int *tc_sticky_flag(Plan &p);  // device copy of that flag kept until reported (or nullptr)

// Process-wide device-memory budget of all plans (fbs_set_device_budget):
// reserve before an allocation (throws FBS_ERR_OOM past the budget), release
// after a free.
void budget_reserve(long long bytes);
void budget_release(long long bytes);

// Transient stream-ordered device buffer counted against the budget; freed
// (on the stream) when it goes out of scope.
struct AsyncBuf {
    void *ptr = nullptr;
    long long bytes = 0;
    cudaStream_t stream = nullptr;
    AsyncBuf(size_t n, cudaStream_t s, const char *what);
    ~AsyncBuf();
    AsyncBuf(const AsyncBuf &) = delete;
    AsyncBuf &operator=(const AsyncBuf &) = delete;
    template <typename T> T *as() const { return reinterpret_cast<T *>(ptr); }
};

}  // namespace fbs
