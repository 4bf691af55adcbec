/*
 * fbs.h -- C ABI of the GB300 FFT polyspectrum estimator.
 *
 * The library computes the binned bispectrum B(k1,k2,k3), power spectrum
 * P(k) and four-shell trispectrum T(k1..k4) of a real periodic N^3 field with
 * the FFT estimator of Watkinson, Majumdar, Pritchard & Mondal (arXiv
 * 1705.06284), Sec. 2:
 *
 *   I_b(n) = sum_{m in S_b} D(m) e^{+2 pi i m.n/N}      shell field   (Eq. delta_nr)
 *   N_b(n) = sum_{m in S_b}      e^{+2 pi i m.n/N}      count field   (Eq. delta_nr)
 *   P_b    = V/N_pix^2   sum_n I_b^2       / sum_n N_b^2            (Eq. Jeong_PS)
 *   B_abc  = V^2/N_pix^3 sum_n I_a I_b I_c / sum_n N_a N_b N_c      (Eq. Jeong_BI)
 *   T_abcd = V^3/N_pix^4 sum_n I_a..I_d    / sum_n N_a..N_d         (Eq. Jeong_gen, p=4)
 *
 * where D(m) = sum_n delta(n) e^{-2 pi i m.n/N} is the unnormalised forward
 * DFT (Eq. DeltaFFTtoDelta), V = L^3 and N_pix = N^3.  Shell b holds the
 * lattice modes m (components wrapped into [-N/2, N/2)) with
 * edges[b] <= |m| k_f < edges[b+1], k_f = 2 pi / L.  sum_n N_a N_b N_c equals
 * N_pix times the exact triangle count N_tri (the denominator of Eq.
 * gen_Nspec3); it is computed once per plan in FP64 and rounded to int64.
 *
 * Everything runs on one CUDA device, on the plan's stream, in hand-written
 * sm_103a kernels.  There is no CPU fallback: without a usable device every
 * entry point that needs one returns FBS_ERR_CUDA.
 *
 * Conventions for every entry point:
 *   - Return FBS_OK (0) or a negative fbs_status; no entry point exits or
 *     aborts.  fbs_last_error() gives a message for the calling thread.
 *   - "Device or host" pointers are classified with cudaPointerGetAttributes:
 *     device (and managed) memory is used in place; host memory (pageable or
 *     pinned) is staged through plan-owned device buffers.  A host field is
 *     copied on a plan-owned copy stream that does not wait for work queued
 *     earlier on the plan's stream (so the copy overlaps it): the host buffer
 *     must hold the field when the call is made, not only once earlier work
 *     on the plan's stream (a device-to-host copy into it, say) completes.
 *   - A plan is not thread-safe: calls on one plan must be serialised by the
 *     caller.  Different plans may be used from different threads.
 */
#ifndef FBS_H
#define FBS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fbs_plan fbs_plan; /* opaque; owns shell tables, counts and workspaces */

typedef enum {
    FBS_OK = 0,
    FBS_ERR_ARG = -1,            /* bad argument (null pointer, edges not ascending, ...) */
    FBS_ERR_UNSUPPORTED_N = -2,  /* N not even, not 2^a 3^b, or outside [8, 512] */
    FBS_ERR_OOM = -3,            /* a device allocation failed */
    FBS_ERR_CUDA = -4,           /* a CUDA call or kernel failed, or no device */
    FBS_ERR_TIMEOUT = -5,        /* a bounded device wait gave up */
    FBS_ERR_STATE = -6,          /* call not valid for this plan (e.g. T on a B-only plan) */
    FBS_ERR_NUMERIC = -7         /* an FP64 count sum was more than 0.25 from an integer */
} fbs_status;

/* Contraction precision (Sec. 2's real-space product sums). FFTs are FP32
 * in every mode; counts are FP64 in every mode. */
enum {
    FBS_PREC_FP32 = 0,    /* CUDA-core FP32 products, FP64 cross-block sums      */
    FBS_PREC_BF16X3 = 1,  /* tcgen05 tensor cores, BF16 hi/lo split, 3 products  */
    FBS_PREC_BF16 = 2     /* tcgen05 tensor cores, plain BF16 (error reported)   */
};

/* Plan flags. */
enum {
    FBS_FLAG_TRISPECTRUM = 1u,   /* also enumerate closed quadruplets (needed by fbs_trispectrum) */
    FBS_FLAG_ALLOW_ALIASED = 2u, /* allow edges beyond N k_f/4 (closure is then modulo N, Sec. 3.2) */
    FBS_FLAG_TIMING = 4u,        /* record CUDA events around every kernel (fbs_plan_kernel_times) */
    FBS_FLAG_FULL_GRID = 8u,     /* evaluate the shell fields and their products on the input
                                    N^3 grid instead of the smallest M^3 grid that gives the same sums */
    FBS_FLAG_SINGLE_GRID = 16u   /* one evaluation grid M > pR for every item (no levels) */
};

/*
 * fbs_plan_create -- build a plan for N^3 fields in a box of side L.
 *   out        : receives the plan (set to NULL on failure).
 *   N          : grid side; even, of the form 2^a 3^b, 8 <= N <= 512.
 *   L          : box side (> 0), physical length units; k_f = 2 pi / L.
 *   edges      : host array of nbins+1 ascending bin edges in physical k units.
 *                Unless FBS_FLAG_ALLOW_ALIASED, edges[nbins] <= N k_f / 4 (every
 *                closed triangle is then closed exactly, not only modulo N,
 *                below the aliasing limit N k_f/3 of Sec. 3.2).
 *   nbins      : 1 <= nbins <= 128.
 *   precision  : FBS_PREC_*.
 *   flags      : FBS_FLAG_* bits.
 *   cuda_stream: cudaStream_t the plan launches on (NULL = legacy default stream).
 * Evaluation grids: the shell field of bin b holds only modes with
 * |m_j| <= R_b, so the product of an item's fields (a triplet or quadruplet)
 * is a trigonometric polynomial of degree <= R_a + R_b + R_c (+ R_d) per axis,
 * and its sum over the N^3 grid equals (N/M)^3 times its sum over any M^3 grid
 * with M above that degree.  The plan groups the items into up to four
 * levels, each an even M = 2^a 3^b <= N above the degree of every item in it
 * (and above 2 R_b of each of its bins), chosen to minimise a work model of
 * the transforms and contractions; each level evaluates only the bins its
 * items use: the same sums up to rounding, with far fewer points than one
 * grid for all.  FBS_FLAG_SINGLE_GRID keeps one level on the smallest
 * M > pR (R the largest component of any bin, p = 3, or 4 with
 * FBS_FLAG_TRISPECTRUM); FBS_FLAG_FULL_GRID and FBS_FLAG_ALLOW_ALIASED keep
 * one level on M = N.  The plan-time count sums use each item's own grid
 * (N_tri = sum_M N_a N_b N_c / M^3).
 * The plan runs the plan-time work on the device before returning: shell
 * tables, the FP64 count fields N_b, exact N_tri (and N_quad) for every
 * candidate bin triple, and the closed-triplet list (lexicographic a<=b<=c
 * with N_tri > 0).  Empty bins give no triplets and P = NaN.
 */
fbs_status fbs_plan_create(fbs_plan **out, int N, double L, const double *edges, int nbins,
                           int precision, unsigned flags, void *cuda_stream);

/*
 * Plan-time counts carried between plans (and processes).  The FP64 count
 * pass of fbs_plan_create depends only on (N, L, edges, flags); a caller that
 * builds the same plan again (a server evicting and re-creating plans, a new
 * process) can skip it:
 * fbs_plan_export_counts -- serialise the plan's closed triplets and
 *   quadruplets with their exact counts into buf (native byte order).  With
 *   buf == NULL only *size is set; otherwise *size is the buffer's capacity on
 *   entry (FBS_ERR_ARG and the needed size when too small) and the bytes
 *   written on return.
 * fbs_plan_create_from_counts -- fbs_plan_create with those results instead
 *   of the count pass.  The blob must come from a plan with the same N, L,
 *   integer bin thresholds and FBS_FLAG_TRISPECTRUM / FBS_FLAG_ALLOW_ALIASED
 *   flags (FBS_ERR_ARG otherwise, no plan).  The plan is the same as one built
 *   from scratch: same items, counts, levels and results.
 */
fbs_status fbs_plan_export_counts(const fbs_plan *plan, void *buf, int64_t *size);
fbs_status fbs_plan_create_from_counts(fbs_plan **out, int N, double L, const double *edges, int nbins,
                                       int precision, unsigned flags, void *cuda_stream, const void *counts,
                                       int64_t size);

/* fbs_plan_free -- release the plan and all its device memory (NULL is a no-op).
 * Synchronises the plan's stream first. */
void fbs_plan_free(fbs_plan *plan);

/* Number of closed triplets (outputs of fbs_bispectrum), or a negative status. */
int fbs_plan_num_triplets(const fbs_plan *plan);

/* Number of closed quadruplets (outputs of fbs_trispectrum; 0 without
 * FBS_FLAG_TRISPECTRUM), or a negative status. */
int fbs_plan_num_quads(const fbs_plan *plan);

/* Copy the closed-triplet table to host arrays: abc[3*ntrip] (int32 bin
 * indices a<=b<=c, lexicographic) and ntri[ntrip] (exact ordered triangle
 * counts).  Either pointer may be NULL. */
fbs_status fbs_plan_triplets(const fbs_plan *plan, int32_t *abc, int64_t *ntri);

/* Copy the closed-quadruplet table: abcd[4*nquad] (a<=b<=c<=d) and
 * nquad_counts[nquad], the ordered quadruple counts (the denominator of Eq.
 * gen_Nspec3 with p = 4) as the nearest FP64 values of the exact counts of
 * fbs_plan_quad_counts_u128 (exact below 2^53).  Either pointer may be NULL. */
fbs_status fbs_plan_quads(const fbs_plan *plan, int32_t *abcd, double *nquad_counts);

/* Exact ordered quadruple counts: words[2*nquad] (host), words[2q] the low
 * and words[2q+1] the high 64 bits of quadruplet q's count as an unsigned
 * 128-bit integer (wide shells on large grids pass 2^63).  Computed at plan
 * time as sum_q C_ab(q) C_cd(q) of integer pair-count convolutions
 * C_ab(q) = #{m1 in S_a, m2 in S_b : m1 + m2 = q}, in integer arithmetic;
 * FBS_ERR_ARG for a NULL argument. */
fbs_status fbs_plan_quad_counts_u128(const fbs_plan *plan, uint64_t *words);

/* Copy shell sizes |S_b| (int64[nbins]) and, if thr != NULL, the integer
 * thresholds on |m|^2 (int64[nbins+1]): bin b holds thr[b] <= |m|^2 < thr[b+1]. */
fbs_status fbs_plan_shells(const fbs_plan *plan, int64_t *sizes, int64_t *thr);

/* Change the contraction precision of an existing plan (FBS_PREC_*). */
fbs_status fbs_plan_set_precision(fbs_plan *plan, int precision);

/* Plan options (fbs_plan_set_option). */
enum {
    FBS_OPT_TC_WIDE = 1, /* 0: tensor-core contraction with the pair products as
                           operand A (M = 128 outer pairs, N = bins; default);
                           1: "wide" orientation with the <= 64 left rows stacked
                           [hi; lo] as operand A and up to 256 right pair
                           products as operand B (BF16x4).  Ignored for FP32. */
    FBS_OPT_TC_ROLES = 2, /* warp roles of the default tensor-core contraction:
                            0 (default) or 1: 16 warps form the pair products
                            and build operand B in turn; 2: 8 warps form the
                            pair products while 8 others build operand B
                            (64-point steps only).  At equal steps the results
                            are identical; only the speed differs (2 measured
                            about 4% slower at 512^3). */
    FBS_OPT_TC_CHUNK = 3, /* points per pipeline step of the default tensor-core
                            contraction: 0 (default) or 2: 128 when two
                            128-column A stages fit beside the accumulators
                            in tensor memory (and 16 product warps are in
                            use), else 64; 1: always 64.  Sums agree within
                            rounding (the CTAs' point ranges differ). */
    FBS_OPT_TC_PAIRS = 4, /* outer rows of the bispectrum's tensor-core
                            contraction: 0 (default): each triplet is carried
                            by one of its three pairs, chosen by a greedy set
                            cover (fewer 128-row tiles); 1: by its pair of
                            the two largest bins (b, c).  Sums agree within
                            rounding. */
    FBS_OPT_SLAB_PLANES = 6,  /* planes of the evaluation grid per slab: 0 (default)
                            the planned slab (as many planes as the slab budget
                            allows); n >= 1: at most n planes per slab (more,
                            thinner slabs in the same buffers).  Sums agree within
                            rounding.  Waits for the plan's stream. */
    FBS_OPT_TC_WAIT_LIMIT = 5 /* clock cycles a warp role of the tensor-core
                            contraction waits for a hand-off from another role
                            before it gives up (0, the default: 2e9 cycles,
                            about one second).  A wait that gives up makes the
                            whole CTA stop issuing work, finish what is in
                            flight (those drain waits keep the default limit),
                            free its tensor memory and return; the evaluation's
                            B and T are then NaN and FBS_ERR_TIMEOUT is
                            reported (see fbs_plan_check).  Meant for testing
                            that path; any value >= 0 is accepted. */,
    FBS_OPT_TC_MERGE = 7      /* BF16x3 products of the tensor-core contraction:
                            0 (default): where the doubled accumulators fit in
                            tensor memory, the hi and lo rows of the inner
                            operand go into one MMA (N = 2 Npad: hi*hi and
                            hi*lo side by side) and lo*hi into a second, two
                            MMAs per K step instead of three; 1: always three.
                            The sums agree within the precision's rounding. */,
    FBS_OPT_TC_BSTAGES = 8    /* shared-memory stages of the tensor-core
                            contraction's inner operand: 0 (default) the first
                            of (B, field) stage depths (4, 4), (3, 4), (2, 4),
                            (3, 2), (2, 2) that fits in shared memory; 2, 3 or
                            4: that many B stages where they fit (else the
                            default).  Sums are identical. */,
    FBS_OPT_TC_BFROMA = 9     /* inner pair rows of the tensor-core contraction
                            (the trispectrum pass's I_a I_b): 0 (default) where
                            the job has one pair tile and every inner pair is
                            also an outer row, the operand-A warps store that
                            product into operand B as well, so operand B is
                            built from the field stage for the single-bin rows
                            only; 1: every inner row is built from the field
                            stage.  Sums are identical. */,
    FBS_OPT_TC_STACK = 10     /* BF16x3 tensor-core contraction of a job with one
                            tile of at most 64 outer pairs: 0 (default) operand
                            A holds the pairs' hi parts in rows 0..63 and their
                            lo parts in rows 64..127, so one MMA per K step
                            (N = 2 Npad) forms hi*hi, hi*lo, lo*hi and lo*lo;
                            1: two MMAs per K step (hi*hi, hi*lo, lo*hi).  The
                            sums agree within the precision's rounding (the
                            stacked form adds the lo*lo products). */
};

/* Set a plan option; FBS_ERR_ARG for an unknown option or value. */
fbs_status fbs_plan_set_option(fbs_plan *plan, int option, int value);

/* Rebind the plan to another cudaStream_t (NULL = legacy default stream). */
fbs_status fbs_plan_set_stream(fbs_plan *plan, void *cuda_stream);

/*
 * fbs_bispectrum -- B for every closed triplet and P for every bin.
 *   field : N^3 FP32 values, C order [x][y][z] (z fastest), device or host.
 *           Caller-owned; read only.
 *   B     : double[ntrip] (device or host), order of fbs_plan_triplets; may be NULL.
 *   P     : double[nbins] (device or host); may be NULL.
 * With device or page-locked (pinned) host outputs the call only enqueues
 * work on the plan's stream and returns: the results are there once the
 * stream reaches them (synchronise it before reading pinned outputs).  With
 * pageable host outputs it synchronises the stream before returning.  A
 * pinned host field is read asynchronously (on the plan's copy stream):
 * leave it unchanged until the plan's stream has passed the call.
 */
fbs_status fbs_bispectrum(fbs_plan *plan, const float *field, double *B, double *P);

/*
 * fbs_bispectrum_batch -- fbs_bispectrum of nfields fields of this plan's grid
 * in one set of launches: every stage (forward transforms, each level's
 * pruned inverse transforms and contraction, the reductions) runs once for
 * all fields, the field taken from a grid dimension, so small grids fill the
 * GPU.  Per field the results equal fbs_bispectrum's (up to rounding: the
 * contraction's point ranges per CTA differ).
 *   fields : host array of nfields DEVICE pointers (N^3 FP32, C order each).
 *   B      : double[nfields * ntrip], field f at B + f*ntrip (device or host).
 *   P      : double[nfields * nbins], field f at P + f*nbins.
 *   nfields: 1 <= nfields, nfields * nbins <= 65535.
 * Bispectra only (no quadruplets).  The first call with a larger nfields than
 * before allocates the batch buffers (plan-owned, kept); the first call with
 * a new list of field pointers uploads it and waits for the stream.  Neither
 * may happen during stream capture; later calls with the same list can be
 * captured.  Same stream semantics as fbs_bispectrum otherwise.
 */
fbs_status fbs_bispectrum_batch(fbs_plan *plan, const float *const *fields, int nfields, double *B, double *P);

/*
 * fbs_trispectrum -- T for every closed quadruplet, plus B and P from the
 * same shell fields (Sec. 2: lower orders come at no extra FFT cost).
 * Needs a plan created with FBS_FLAG_TRISPECTRUM (else FBS_ERR_STATE).
 * T: double[nquad]; B: double[ntrip]; P: double[nbins]; each device or host
 * or NULL.  Same stream semantics as fbs_bispectrum.  The estimator is the
 * raw p = 4 form (no subtraction of disconnected parts).
 */
fbs_status fbs_trispectrum(fbs_plan *plan, const float *field, double *T, double *B, double *P);

/*
 * fbs_trispectrum_connected -- the connected trispectrum Tc of every closed
 * quadruplet, with T, B and P of the same evaluation (FBS_FLAG_TRISPECTRUM
 * plans).  The paper's four-shell estimator (Eq. Jeong_gen with p = 4) sums
 * every closed quadruple of modes; for shells a = b, c = d that includes the
 * paired quadruples (m1 + m2 = 0, or another pair of modes summing to zero),
 * whose terms |D(m1)|^2 |D(m3)|^2 carry the disconnected P x P part of the
 * four-point function.  Tc leaves every paired quadruple out:
 *   Tc = V^3/N_pix^4 (sum_n I_a I_b I_c I_d / N_pix - paired sum) / N_conn
 * with the paired sum from per-shell sums over the spectrum (inclusion-
 * exclusion over the three pairings; a = b < c = d: S2_a S2_c, a = b = c = d:
 * 3 S2^2 - 3 S4 + the self-conjugate modes' D^4, S2/S4 the shell's sums of
 * |D|^2 and |D|^4) and N_conn the unpaired count (fbs_plan_quads_connected).
 * A Gaussian field's Tc has zero mean.  Tc is NaN where a quadruplet has no
 * unpaired quadruple.  Tc[nquad], T[nquad], B[ntrip], P[nbins]: device or
 * host or NULL; same stream semantics as fbs_bispectrum.
 */
fbs_status fbs_trispectrum_connected(fbs_plan *plan, const float *field, double *Tc, double *T, double *B,
                                     double *P);

/*
 * fbs_plan_tc_info -- diagnostics of level `level`'s tensor-core job `which`
 * (0: triplets, 1: quadruplets, 2: the fused triplet + quadruplet pass),
 * available after an evaluation has built it: info[11] = {built, usable,
 * outer 128-row tiles of the largest CTA group, inner rows, inner rows padded
 * (N of the MMA), 1 when the latest launch put the hi and lo rows in one MMA
 * (FBS_OPT_TC_MERGE), 2 when it also stacked operand A's hi and lo rows on M
 * (FBS_OPT_TC_STACK), else 0 (-1 before any launch), 64-point K-atoms per
 * pipeline step of that launch, its operand-A stages in tensor memory, its
 * operand-B stages and its field stages in shared memory, the number of
 * inner pair rows it took from operand A (FBS_OPT_TC_BFROMA; 0: none)}.
 * FBS_ERR_ARG for a bad level or job.
 */
fbs_status fbs_plan_tc_info(const fbs_plan *plan, int level, int which, int32_t *info);

/*
 * fbs_plan_follow -- make `follower` evaluate the spectrum of `leader`'s most
 * recent evaluation instead of transforming a field of its own: one field
 * upload and one forward transform serve both plans (a bispectrum plan and a
 * trispectrum plan of the same field, say).  Requirements (FBS_ERR_ARG /
 * FBS_ERR_STATE otherwise): the same grid N, a leader spectrum box at least
 * as large as the follower's (top edge at least as high), the same stream
 * (the follower's kernels are ordered after the leader's forward transform
 * and before its next one by the stream), and a leader that does not follow
 * another plan.  A following plan's evaluation calls take field = NULL
 * (a non-NULL field is FBS_ERR_STATE) and read the leader's box as the
 * leader's last call on the stream left it.  The leader must outlive the
 * follower or be detached first: leader = NULL restores the follower's own
 * box.  Batched evaluations (fbs_bispectrum_batch) are not affected.
 */
fbs_status fbs_plan_follow(fbs_plan *follower, const fbs_plan *leader);

/*
 * Diagonal-resolved trispectrum (FBS_FLAG_TRISPECTRUM plans).  Every closed
 * quadruple (m1, m2, m3, m4) of quadruplet (a <= b <= c <= d) has the
 * diagonal q = m1 + m2 = -(m3 + m4) of its quadrilateral; the diagonal bins
 * split the quadruples by |q| into shells diag_edges[D] <= |q| k_f <
 * diag_edges[D+1] (the same integer-threshold rule as the bins; an edge of 0
 * admits q = 0, the paired quadruples m2 = -m1 of a = b, c = d):
 *   T_D = V^3/N_pix^4 num_D / N_D,
 *   num_D = sum_{q in S_D} F_ab(q) F_cd(-q),  F_ab(q) = sum_{m1 + m2 = q} D(m1) D(m2),
 *   N_D   = sum_{q in S_D} C_ab(q) C_cd(-q),  C_ab(q) = #{m1 + m2 = q}.
 * Over diagonal shells that cover every |q|, the num_D and N_D add up to the
 * four-shell sum and count of Eq. Jeong_gen (p = 4).
 *
 * fbs_plan_set_diagonal -- set ndiag >= 1 diagonal bins (host array
 * diag_edges[ndiag+1], ascending, physical k units) and compute the exact
 * counts N_D at plan time (FP64 count fields and integer pair counts, as the
 * quadruple counts).  May be called again; the device tables of an earlier
 * call are released with the plan.  FBS_ERR_STATE without FBS_FLAG_TRISPECTRUM.
 * fbs_plan_num_diagonal_bins -- ndiag, 0 before fbs_plan_set_diagonal.
 * fbs_plan_diagonal_counts -- counts[nquad*ndiag] as FP64 (nearest double)
 * and/or words[2*nquad*ndiag] as unsigned 128-bit integers (low, high),
 * quadruplet-major; either may be NULL.
 * fbs_trispectrum_diagonal -- TD[nquad*ndiag] (quadruplet-major, NaN where
 * N_D = 0) of one field (device or host, as fbs_bispectrum).  The shell
 * fields of each level are held on the whole evaluation grid at once (bins x
 * M^3 FP32), the products I_a I_b of the distinct first and second pairs of
 * the quadruplets are forward transformed on that grid (FP32), and num_D is
 * accumulated in FP64 over the half spectrum.  TD: device or host.
 */
fbs_status fbs_plan_set_diagonal(fbs_plan *plan, const double *diag_edges, int ndiag);
int fbs_plan_num_diagonal_bins(const fbs_plan *plan);
fbs_status fbs_plan_diagonal_counts(const fbs_plan *plan, double *counts, uint64_t *words);
fbs_status fbs_trispectrum_diagonal(fbs_plan *plan, const float *field, double *TD);

/*
 * Non-cubic grids and complex fields (Sec. 2: its footnote on non-cubic data,
 * and the remark that Eq. Jeong_gen applies to complex data through complex
 * DFTs).  A separate plan type on the whole grid, FP32 transforms and
 * products with FP64 sums, bispectrum and power spectrum.
 *
 * fbs_gplan_create -- grid n[3] = (N_x, N_y, N_z), each 2^a 3^b in 2..512;
 * box L[3] = (L_x, L_y, L_z) > 0; edges[nbins+1] ascending, physical k.  Mode
 * m (components in FFT order) has k = 2 pi (m_x/L_x, m_y/L_y, m_z/L_z) and is
 * in bin b when t_b <= s(m) < t_{b+1}, s(m) = (m_x/L_x)^2 + (m_y/L_y)^2 +
 * (m_z/L_z)^2 and t_b = (edges[b] / 2 pi)^2 (FP64, in that order).  Closed
 * triplets a <= b <= c close modulo the grid along each axis; unless flags
 * holds FBS_FLAG_ALLOW_ALIASED every mode of every bin must have |m_j| <
 * N_j/4 (FBS_ERR_ARG otherwise), where that is exact closure.  Exact
 * triangle counts from FP64 count fields at plan time (FBS_ERR_NUMERIC if a
 * count sum is not within 0.25 of an integer).  Other flags are ignored.
 * fbs_gplan_num_triplets / fbs_gplan_triplets (abc[3*ntrip], ntri[ntrip],
 * either may be NULL) / fbs_gplan_shells (sizes[nbins]) -- host copies.
 * fbs_gplan_bispectrum -- field: complex64 interleaved (re, im) floats,
 * [N_x][N_y][N_z], device or host (a real field: imaginary parts zero).
 * B[2*ntrip] = (Re, Im) of V^2/N_pix^3 sum_n I_a I_b I_c / (N_pix N_tri) and
 * P[2*nbins] = (Re, Im) of V/N_pix^2 sum_n I_b I_b / (N_pix |S_b|) (NaN for
 * empty bins), V = L_x L_y L_z, N_pix = N_x N_y N_z, I_b the unnormalised
 * inverse DFT of the spectrum on S_b; device or host, either may be NULL.
 * Synchronous (returns with the outputs written).
 * fbs_gplan_free -- releases the plan (NULL is a no-op).
 */
typedef struct fbs_gplan fbs_gplan;
fbs_status fbs_gplan_create(fbs_gplan **out, const int32_t *n, const double *L, const double *edges, int nbins,
                            uint32_t flags);
int fbs_gplan_num_triplets(const fbs_gplan *g);
fbs_status fbs_gplan_triplets(const fbs_gplan *g, int32_t *abc, int64_t *ntri);
fbs_status fbs_gplan_shells(const fbs_gplan *g, int64_t *sizes);
fbs_status fbs_gplan_bispectrum(fbs_gplan *g, const float *field, double *B, double *P);
void fbs_gplan_free(fbs_gplan *g);

/*
 * fbs_plan_triangle_average -- a model averaged over each closed triplet's
 * exact set of triangles, as the paper compares theory with its measurements
 * (theory evaluated for every triangle contributing to a bin and averaged,
 * Sec. 3.3): for triplet (a <= b <= c),
 *   out[t] = (1/N_tri) sum over ordered closed (m1, m2, m3) in S_a x S_b x S_c
 *            of sum_k coef[k] f_{terms[3k]}(|m1|) f_{terms[3k+1]}(|m2|) f_{terms[3k+2]}(|m3|).
 * Models whose bispectrum is a sum of such separable terms (a product of
 * functions of k1, k2, k3 each) are covered exactly: the local-type
 * 2 f (P1 P2 + cyc), the equal-radius bubble model's W(k1 R) W(k2 R) W(k3 R)
 * (Eq. BharBk), and tree-level perturbation theory (Eq. PT_Bi), whose kernel
 * is a polynomial in k1.k2 = (k3^2 - k1^2 - k2^2)/2 over powers of k1 k2.
 * By the Kronecker-delta identity of Sec. 2 each term is the FP64 sum over the
 * evaluation grid of three weighted count fields (the inverse transforms of
 * f(|m|) on the shells, the count fields of Eq. delta_nr with weights), so
 * no triangle is enumerated.
 *   w     : host double[nfunc * nw]; f_i(|m|) tabulated at integer |m|^2 = s,
 *           w[i*nw + s], nw >= the plan's top threshold (fbs_plan_shells).
 *   terms : host int32[3 * nterms], function of each position; coef: host double[nterms].
 *   out   : host double[ntrip], the order of fbs_plan_triplets.
 * Synchronous; allocates FP64 fields for the functions in use (transient).
 */
fbs_status fbs_plan_triangle_average(fbs_plan *plan, const double *w, int nfunc, int64_t nw, const int32_t *terms,
                                     const double *coef, int nterms, double *out);

/* Average of w(|m|) over the modes of each bin: out[b] = sum_{m in S_b}
 * w[|m|^2] / |S_b| (NaN for empty bins); w tabulated at integer |m|^2 up to
 * at least the top threshold (nw).  Host computation. */
fbs_status fbs_plan_shell_average(const fbs_plan *plan, const double *w, int64_t nw, double *out);

/* Unpaired ordered quadruple counts N_conn[nquad] of the connected
 * trispectrum (FP64; exact integers where the quadruple counts are). */
fbs_status fbs_plan_quads_connected(const fbs_plan *plan, double *nconn);

/*
 * fbs_plan_sums -- the raw FP64 real-space sums of the last call, for
 * diagnostics and tests: num_trip[ntrip] = sum_n I_a I_b I_c,
 * num_quad[nquad] = sum_n I_a I_b I_c I_d, sumsq[nbins] = sum_n I_b^2.  Host
 * arrays (any may be NULL); synchronises the stream.
 */
fbs_status fbs_plan_sums(fbs_plan *plan, double *num_trip, double *num_quad, double *sumsq);

/*
 * fbs_plan_check -- wait for the plan's stream and report whether an
 * evaluation since the last report gave up a tensor-core wait
 * (FBS_ERR_TIMEOUT; the outputs of that evaluation are NaN).  The report is
 * given once and then cleared.  Asynchronous callers (device or pinned
 * outputs) learn of a timeout here, from fbs_plan_sums, or from a later
 * fbs_bispectrum / fbs_trispectrum: an estimator call first checks, without
 * waiting, whether an earlier evaluation on the plan is already known to have
 * timed out, and if so returns FBS_ERR_TIMEOUT without enqueuing anything
 * (the check is skipped while the plan's stream is being captured).
 * Calls with pageable host outputs wait for their results and report a
 * timeout directly.
 */
fbs_status fbs_plan_check(fbs_plan *plan);

/*
 * fbs_set_device_budget -- process-wide cap (bytes) on the device memory all
 * plans together may hold, plan-time scratch included (0, the default: no
 * cap).  An allocation that would pass the cap fails as a failed cudaMalloc
 * does: the call returns FBS_ERR_OOM and a failed fbs_plan_create leaves no
 * plan and no memory behind.  Existing plans are not affected by lowering it.
 * fbs_device_bytes_in_use -- bytes the library's plans hold now.
 */
fbs_status fbs_set_device_budget(int64_t bytes);
int64_t fbs_device_bytes_in_use(void);

/*
 * fbs_set_slab_budget -- process-wide default (bytes) of the shell-field slab
 * buffer of plans created after the call (0 restores the default, 8 GiB; the
 * environment variable FBS_SLAB_MB, when set, takes precedence).  A smaller
 * slab holds fewer planes of the evaluation grid at once: less memory per
 * plan (a server keeps more plans resident), more launches per evaluation.
 * FBS_ERR_ARG for a negative value.
 */
fbs_status fbs_set_slab_budget(int64_t bytes);

/*
 * fbs_plan_kernel_times -- with FBS_FLAG_TIMING, the CUDA-event time (ms) and
 * launch count accumulated per kernel class since the last reset, in the
 * order of fbs_kernel_class_name(0..n-1).  ms and launches are host arrays of
 * n entries (n = fbs_num_kernel_classes()).  reset != 0 zeroes the counters
 * after reading.  Synchronises the stream.
 */
int fbs_num_kernel_classes(void);
const char *fbs_kernel_class_name(int i);
fbs_status fbs_plan_kernel_times(fbs_plan *plan, double *ms, int64_t *launches, int reset);

/* Plan-time cost (ms of wall time spent in fbs_plan_create). */
double fbs_plan_create_ms(const fbs_plan *plan);

/* Largest distance of sum_n N_a N_b N_c / N_pix from the nearest integer over
 * all candidate triples at plan time (FP64 rounding diagnostics; the plan
 * fails with FBS_ERR_NUMERIC when it exceeds 0.25). */
double fbs_plan_count_margin(const fbs_plan *plan);

/* 1 for a plan (its quadruple counts are exact integers, see
 * fbs_plan_quad_counts_u128), <0 on error. */
int fbs_plan_quad_counts_exact(const fbs_plan *plan);

/* Side M of the largest evaluation grid of the plan (its last level). */
int fbs_plan_eval_grid(const fbs_plan *plan);

/* Planes per slab of that level's grid (the shell fields of one slab are
 * resident at a time; slabs are balanced, the last may be shorter) and its
 * number of slabs per evaluation; <0 on error. */
int fbs_plan_slab_planes(const fbs_plan *plan);
int fbs_plan_num_slabs(const fbs_plan *plan);

/* Number of evaluation levels (grids ascending), or <0 on error. */
int fbs_plan_num_levels(const fbs_plan *plan);

/* Level i (0 <= i < fbs_plan_num_levels): its grid M, the bins it evaluates,
 * the closed triplets and quadruplets it contracts, and its slab planes and
 * slabs per evaluation.  Any output pointer may be NULL. */
fbs_status fbs_plan_level(const fbs_plan *plan, int i, int *M, int *nbins, int *ntrip, int *nquad,
                          int *slab_planes, int *nslabs);

/* The level of every closed triplet (trip_level[ntrip], order of
 * fbs_plan_triplets) and quadruplet (quad_level[nquad]); either may be NULL. */
fbs_status fbs_plan_item_levels(const fbs_plan *plan, int32_t *trip_level, int32_t *quad_level);

/* Device bytes owned by the plan. */
int64_t fbs_plan_device_bytes(const fbs_plan *plan);

/*
 * fbs_triple_sums_noalloc -- num[t] = sum_{p < npts} f_a[p] f_b[p] f_c[p] for
 * (a, b, c) = abc[3t..3t+2], without allocating any device memory.
 *
 * The paper has no counterpart: this is for callers that already hold real
 * fields on the device (for instance shell fields made by their own code) and
 * cannot call cudaMalloc, because their device memory belongs to another
 * allocator that must account for every byte, or because the process reserves
 * all device memory up front.  The caller passes every input and output; the
 * per-block FP64 partial sums live in a static device array of 152 x 4096
 * doubles (4.75 MiB) that each GPU loading the library holds until exit.
 *   fields    : device FP32, nfields fields, field i at fields + i*bin_stride.
 *   nfields   : >= 1; triplet entries outside [0, nfields) give NaN sums.
 *   bin_stride: elements between fields (>= npts).
 *   npts      : points summed per field.
 *   abc       : device int32[3*ntrip].
 *   ntrip     : 0 <= ntrip <= 4096 (larger: FBS_ERR_ARG, nothing launched).
 *   num       : device double[ntrip], written (FP32 products in runs of 64
 *               terms, FP64 across runs and blocks, fixed reduction order).
 *   cuda_stream: stream of both launches (NULL = legacy default stream).
 * Asynchronous on the stream.  The first call on a device looks up the
 * scratch array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  The address is
 * kept for the life of the process: do not use this entry point after a
 * cudaDeviceReset (or another teardown of the device's primary context) in
 * the same process, because the array may then sit elsewhere.  All calls share
 * the one scratch array, which keeps the last call's partials: calls that
 * overlap on the GPU (different streams, different host threads) race, so
 * serialise them.  Returns FBS_OK, FBS_ERR_ARG or FBS_ERR_CUDA.
 */
fbs_status fbs_triple_sums_noalloc(const float *fields, int nfields, long long bin_stride,
                                   long long npts, const int32_t *abc, int ntrip, double *num,
                                   void *cuda_stream);

/*
 * Fine bins, then (k1, k2, cos theta) cells.  The paper advises measuring with
 * one-pixel bins and binning further afterwards (Sec. 3.1), and shows the
 * bispectrum against theta, the triangle's internal angle between k1 and k2
 * (k3 = -k1 - k2 closes it):  cos theta = (k1^2 + k2^2 - k3^2) / (2 k1 k2),
 * clamped to [-1, 1] (the representative sides of a closed triplet can break
 * the triangle inequality by up to a bin width: the degenerate end).
 * A rebin regroups a plan's closed triplets: each distinct assignment of a
 * triplet's three bins to the sides (k1, k2, k3), with the bins'
 * representative k, is one configuration; a cell (K1, K2, MU) collects the
 * ordered closed triples (count N_tri, FP64 sum) of every configuration with
 * k1 in k bin K1, k2 in k bin K2 and cos theta in bin MU, and its estimate is
 * the direct estimator over that union of triangle sets:
 *   B_cell = V^2/N_pix^3 sum num / (N_pix sum N_tri)    (Eq. bi_direct).
 *
 * fbs_rebin_create
 *   plan     : the fine-bin plan (its closed triplets are read; the rebin stays
 *              valid while the plan lives).
 *   k_rep    : host double[nbins], the k of each fine bin (physical units), or
 *              NULL for the midpoint of each bin's edges.
 *   k_edges  : host double[nk+1] ascending, the cells' k bins (both k1 and k2).
 *   mu_edges : host double[nmu+1] ascending, the cells' cos theta bins.
 *   Cells are ordered (K1 * nk + K2) * nmu + MU; nk * nk * nmu <= 2^26.
 *   Configurations outside the edges are left out.
 * fbs_rebin_bispectrum -- after an evaluation on the plan (fbs_bispectrum or
 *   fbs_trispectrum): B[nk*nk*nmu] (device or host; NaN for empty cells), on
 *   the plan's stream, with the same stream semantics as fbs_bispectrum.
 * fbs_rebin_counts -- ordered triple count of every cell (host int64).
 * fbs_rebin_free -- release it (NULL is a no-op).
 */
typedef struct fbs_rebin fbs_rebin;
fbs_status fbs_rebin_create(fbs_rebin **out, const fbs_plan *plan, const double *k_rep, const double *k_edges,
                            int nk, const double *mu_edges, int nmu);
fbs_status fbs_rebin_bispectrum(fbs_rebin *rebin, fbs_plan *plan, double *B);
fbs_status fbs_rebin_counts(const fbs_rebin *rebin, int64_t *counts);
void fbs_rebin_free(fbs_rebin *rebin);

/* Message of the last failure on the calling thread ("" if none). */
const char *fbs_last_error(void);

/* ABI version (major*100 + minor). */
int fbs_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FBS_H */
