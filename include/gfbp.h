/*
 * gfbp — belief-propagation decoding of LDPC codes over GF(q), q = 2^p <= 256,
 * on one NVIDIA GB300 (sm_103a).
 *
 * Method: N. Yacov, H. Efraim, H. Kfir, I. Kanter, O. Shental, "Parallel vs.
 * Sequential Belief Propagation Decoding of LDPC Codes over GF(q) and Markov
 * Sources" (arXiv cs/0605069).  Section and equation numbers are the paper's.
 *
 * Conventions shared by every entry point
 *   - Symbols are GF(2^p) elements 0..q-1; bit k of symbol a is (a >> k) & 1;
 *     GF addition is XOR (Sec. 2: "r = t + n mod 2" on the binary image).
 *   - Edges of H are ordered by (row, col); every per-edge array uses that order.
 *   - "device" pointers are CUDA global-memory addresses of the current device;
 *     "host" pointers are ordinary CPU memory.  The caller owns every buffer it
 *     passes; the library keeps no pointer to caller memory after the call's
 *     work on `stream` has completed.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls are
 *     stream-ordered and asynchronous unless stated otherwise.
 *   - Errors: every call returns a status.  Arguments are validated on the host
 *     before any launch; on error nothing is launched and gfbp_last_error()
 *     describes the cause.  No kernel traps; device-side anomalies are reported
 *     through status words.
 */
#ifndef GFBP_H
#define GFBP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GFBP_OK = 0,
    GFBP_EINVAL = 1,      /* invalid argument (reason in gfbp_last_error) */
    GFBP_ENOMEM = 2,      /* host or device allocation failed */
    GFBP_ECUDA = 3,       /* a CUDA runtime call failed */
    GFBP_ETIMEOUT = 4,    /* a bounded wait ran out */
    GFBP_EBUSY = 5,       /* resource in use (e.g. a full admission budget) */
    GFBP_EUNSUPPORTED = 6 /* valid input outside what this build implements */
} gfbp_status;

/* Thread-local description of the last error of this thread's calls. */
const char* gfbp_last_error(void);

/* ------------------------------------------------------------------ code */
typedef struct gfbp_code gfbp_code; /* opaque; owns a device copy of H */

/*
 * Build a code from the sparse parity-check matrix H (M x N) over GF(q)
 * (Sec. 2: the non-zero elements of row i are the symbols of check i, those of
 * column j the checks of symbol j; non-zero values are in {1..q-1}).
 *   q          field size, 2^p with 1 <= p <= 8.
 *   M, N       rows (checks) and columns (symbols); N >= 1, M >= 0.
 *   nnz        number of non-zeros E.
 *   row, col, val  host [nnz] COO triplets, 0 <= row < M, 0 <= col < N,
 *              1 <= val < q, no duplicate (row, col); any order (the library
 *              sorts by (row, col)).
 *   prim_poly  field polynomial with bit k = coefficient of x^k (degree p, must
 *              be primitive); 0 = default x^2+x+1, x^3+x+1, x^4+x+1, x^5+x^2+1,
 *              x^6+x+1, x^7+x^3+1, x^8+x^4+x^3+x^2+1.
 *   out        receives the handle.
 * Synchronous: copies H to the current device before returning.  Row degree
 * must be <= 16 and column degree <= 8 (GFBP_EUNSUPPORTED otherwise).
 */
gfbp_status gfbp_code_create(int32_t q, int32_t M, int32_t N, int64_t nnz, const int32_t* row,
                             const int32_t* col, const int32_t* val, uint32_t prim_poly, gfbp_code** out);

/* Release a code (synchronous; no decode using it may still be in flight). */
void gfbp_code_destroy(gfbp_code* code);

/*
 * The SUS level schedule that gfbp_code_create builds for H, computed on the
 * host alone (no device needed; for inspection and tests).  Column j's level
 * is 0 when it shares no check with an earlier column, else 1 + the highest
 * level of those columns, so the columns of one level share no check and
 * updating the levels in turn, a level's columns at once, gives every column
 * the operands of the sequential order of Sec. 2.  The levels are cut into
 * pieces: runs of whole columns of one level (columns increasing), at most
 * 128 (column, slot) pairs each, a column without checks counting as one
 * pair (slot 0).  Inside a piece the pairs are listed in the order the q <= 16
 * level kernel takes them: first those at an inner position of their check
 * (1..d_c-2), then those at position 0, then the rest; pair_row is the pair's
 * index in the piece's column order (a column's slots have consecutive rows).
 *   q, M, N, nnz, row, col, val  as gfbp_code_create (same validation, errors).
 *   level      host [N] out.
 *   n_levels   out: 1 + the highest level.
 *   piece_ptr  host [nnz + N + 1] out: pair offsets of the pieces; n_pieces + 1 written.
 *   pair_col, pair_slot, pair_row  host [nnz + N] out; n_pairs written.
 */
gfbp_status gfbp_level_schedule(int32_t q, int32_t M, int32_t N, int64_t nnz, const int32_t* row, const int32_t* col,
                                const int32_t* val, int32_t* level, int32_t* n_levels, int32_t* piece_ptr,
                                int32_t* n_pieces, int32_t* pair_col, int32_t* pair_slot, int32_t* pair_row,
                                int32_t* n_pairs);

/* Sizes of a code; any output pointer may be NULL. */
gfbp_status gfbp_code_info(const gfbp_code* code, int32_t* q, int32_t* M, int32_t* N, int64_t* E,
                           int32_t* max_row_degree, int32_t* max_col_degree);

/* ------------------------------------------------------------- decoding */
typedef enum {
    GFBP_BSC = 0,    /* obs [F][N][p] bits 0/1; param = flip rate f          */
    GFBP_BEC = 1,    /* obs [F][N][p] bits 0/1, 2 = erased; param unused      */
    GFBP_BIAWGN = 2, /* obs [F][N][p] real y, BPSK bit 0 -> +1; param = sigma */
    GFBP_LOGLIK = 3  /* obs [F][N][q] log-likelihood of every symbol          */
} gfbp_channel_kind;

typedef struct {
    int32_t kind;             /* gfbp_channel_kind */
    float param;              /* f (BSC), sigma (BI-AWGN); ignored otherwise */
    const float* frame_param; /* optional device [F]: per-frame param (overrides param) */
} gfbp_channel;

typedef enum { GFBP_PUS = 0, GFBP_SUS = 1 } gfbp_schedule;

typedef enum { GFBP_PRIOR_IID = 0, GFBP_PRIOR_MARKOV = 1, GFBP_PRIOR_MARKOV_GS = 2 } gfbp_prior_kind;

/*
 * Source prior (Sec. 2).  I.i.d.: Pr(s = a) = 1/q for every symbol.  Markov:
 * dynamical block priors re-estimated after every iteration by Eq. 6-7 from
 * the pseudo-posteriors of the neighbouring source symbols; every other symbol
 * keeps the uniform prior.
 * MARKOV_GS (a variant the paper leaves open; SUS with gfbp_decode only): the
 * block prior of source symbol i is re-estimated by Eq. 6 just before the
 * sweep reaches its column, from its neighbours' pseudo-posteriors as they
 * stand at that moment (this sweep's where the sweep has passed them, the
 * previous sweep's otherwise; before a symbol's first visit, its initial
 * belief: channel likelihood times the stationary distribution, normalised),
 * and not between sweeps.  The sweep is then a chain through the source
 * symbols, so it runs on the column-walking kernel (a lane group per frame;
 * q <= 16, or the TRANSFORM check method for q >= 32).  PUS, gfbp_step,
 * batches and the server return GFBP_EUNSUPPORTED for it.
 */
typedef struct {
    int32_t kind;           /* gfbp_prior_kind */
    const double* T;        /* host [q][q] transition matrix, T[a][b] = Pr(next = b | a);
                               rows are renormalised to sum 1 */
    int32_t K;              /* number of source symbols, 1 <= K <= N */
    const int32_t* src_pos; /* host [K] distinct symbol positions in source order;
                               NULL = 0..K-1 */
} gfbp_prior;

/*
 * Arithmetic of the horizontal pass (Eq. 3).  Both compute the same r_ij:
 *   TRANSFORM  the XOR-convolution theorem: Walsh-Hadamard transforms of the
 *              relabelled messages, pointwise product, inverse transform; stored
 *              as mode-shifted deviations formed with additions only (any q).
 *              Entries far below the largest keep an absolute error of about
 *              1e-7 of the largest.
 *   DIRECT     the configuration sum by successive XOR-convolutions of the
 *              relabelled messages, non-negative arithmetic only, every entry
 *              to relative precision (any q; q^2 FMAs per convolution, in
 *              registers for q <= 16, from shared memory by lane groups for
 *              q >= 32).
 *   TENSOR     the convolution theorem with plain transforms stored (F =
 *              WHT of the relabelled q), the transforms inside the sweep taken
 *              as dense +-1 Hadamard contractions on the tensor cores (FP16
 *              hi/lo split of power-of-two-scaled vectors, FP32 accumulation;
 *              gfbp_wht).  SUS only, q >= 16; posteriors within 1e-4 of the
 *              FP64 oracle per iteration (tested).
 *   AUTO       DIRECT for q <= 64 (posteriors within 1e-5 of the FP64 oracle
 *              per iteration, tested), TRANSFORM for q = 128, 256, where
 *              DIRECT's q^2 FMAs per convolution (65536 at q = 256) make long
 *              decodes impractical; DIRECT stays available there (within 1e-5,
 *              tested).  TENSOR is an explicit choice.
 */
typedef enum {
    GFBP_CHECK_AUTO = 0,
    GFBP_CHECK_TRANSFORM = 1,
    GFBP_CHECK_DIRECT = 2,
    GFBP_CHECK_TENSOR = 3
} gfbp_check_method;

/*
 * How the kernels for q <= 16 with the DIRECT check node hold a q-vector.
 * Both layouts give the same bits (for SUS with q >= 4; at q = 2 the lane
 * layout runs the generic group kernel, whose sums run in another order).
 *   LANES   spread over a group of lanes.  PUS: a lane group per check and
 *           per column.  SUS: lane teams walk the columns in order; with
 *           sus_width > 1 teams per frame, a column starts once the last
 *           earlier column sharing a check with it is done (column degree
 *           <= 4, row degree <= 8).
 *   THREAD  in one thread's registers.  PUS: a thread per check and per
 *           column.  SUS: the columns are grouped into levels (level(j) = 1 +
 *           the highest level of the earlier columns sharing a check with j;
 *           one level's columns share no check) and a level's (column, check)
 *           pairs run at once, a thread each.
 *   RESIDENT  THREAD's arithmetic with the frame's whole edge slab held in
 *           one CTA's shared memory from the first iteration to the last
 *           (E q 4 bytes plus about 10 KB must fit the opt-in shared memory
 *           of a CTA, 227 KB on GB300: GF(16) up to about 3,500 edges).  The
 *           messages never travel to global memory; a sweep reads only the
 *           frame's channel likelihoods and block priors.  PUS: the bits of
 *           THREAD (row degree <= 6, column degree <= 4).  SUS: the bits of
 *           THREAD with RUNNING partials (the partial convolutions replace
 *           the check's messages in their own slots), so sus_partials must be
 *           AUTO or RUNNING.  GFBP_EUNSUPPORTED where it does not apply.
 *   L2RESIDENT  (SUS) RESIDENT's kernel and bits with each CTA's slab in
 *           the workspace instead of shared memory, and only as many CTAs at
 *           once as keep all their slabs within 75% of the L2 (several per
 *           SM for GF(16), N = 1000), so that the messages stay on chip and
 *           the CTAs' latencies overlap; any code size (q <= 16).
 *   AUTO    PUS: RESIDENT where it applies, else THREAD; SUS: RESIDENT up
 *           to 4 frames per SM (AUTO partials; where one frame's latency
 *           sets the time), else THREAD, whose many frames per SM hide each
 *           other's latency (PUS THREAD measured against
 *           LANES: 10% faster on GF(16), N = 1000; 18% on GF(8), N = 2000;
 *           2.9x on GF(4), N = 96).
 * SUS with the TRANSFORM check node (any q) also runs by levels unless LANES
 * is asked for: a lane group per (column, check) pair instead of per frame,
 * the same bits as the lane kernel.
 */
typedef enum {
    GFBP_LAYOUT_AUTO = 0,
    GFBP_LAYOUT_LANES = 1,
    GFBP_LAYOUT_THREAD = 2,
    GFBP_LAYOUT_RESIDENT = 3,
    GFBP_LAYOUT_L2RESIDENT = 4
} gfbp_layout;

/*
 * How the SUS level kernel (THREAD layout, DIRECT check node, q <= 16)
 * gathers a check's other messages (Eq. 3) when it visits column j.  When the
 * sweep reaches j, the check's messages from columns before j already hold
 * this sweep's values and those from columns after j still hold the values
 * the sweep started with.
 *   FOLD     every visit convolves the check's d_c - 1 other messages afresh
 *            (d_c - 2 convolutions per visit); the lane kernels' arithmetic,
 *            bit for bit.
 *   RUNNING  at the start of each sweep the suffix convolutions of every
 *            check's messages (positions m..d_c-1, m >= 1) are formed at once;
 *            during the sweep each check keeps the convolution of its messages
 *            updated so far.  A visit then takes at most one convolution for r
 *            and one to extend the prefix: about half the arithmetic of FOLD.
 *            The same r up to the order of FP32 operations.  A frame's partials
 *            sit in shared memory (E q 4 bytes; a CTA of q/4 threads per pair
 *            per frame: GF(16) up to about 3,300 edges); where they do not
 *            fit, FOLD runs instead.
 *   RUNNING_GLOBAL  the same arithmetic with the partials in global memory
 *            (a second edge slab, F E q 4 bytes, allocated stream-ordered by
 *            the call itself; refused by gfbp_decode_noalloc): the same bits
 *            as RUNNING.
 *   AUTO     RUNNING up to 4 frames per SM (with layout AUTO the frame's
 *            partials in shared memory, the RESIDENT kernel: GF(16), N =
 *            1000, 20 iterations, 152 frames 1.49 ms against 2.41 ms for
 *            FOLD), FOLD above (with many frames resident per SM their
 *            latencies overlap: 4096 frames 19.6 ms against 24.5 ms).  The
 *            choice follows the frame count, so a frame's posteriors can
 *            differ in the last bits between a call with few frames and one
 *            with many; FOLD or RUNNING fix the kernel and with it the bits.
 * Other kernels ignore the option.
 */
typedef enum {
    GFBP_PARTIALS_AUTO = 0,
    GFBP_PARTIALS_FOLD = 1,
    GFBP_PARTIALS_RUNNING = 2,
    GFBP_PARTIALS_RUNNING_GLOBAL = 3
} gfbp_sus_partials;

/* Optional inputs and outputs of gfbp_decode / gfbp_step (NULL = defaults). */
typedef struct {
    const uint8_t* punct;    /* device [N]: 1 = symbol not observed (uniform likelihood) */
    const uint8_t* syndrome; /* device [F][M]: decode H x = z (Eq. 2); NULL = z = 0 */
    float* post;             /* device [F][N][q]: pseudo-posteriors Q (Eq. 5) at the end */
    uint8_t* xhat_trace;     /* device [F][max_iter][N]: hard decisions after every
                                iteration, 255 after the frame stopped (decode only) */
    int32_t no_early_stop;   /* nonzero: run max_iter iterations even after H x = z */
    void* workspace;         /* device scratch of >= gfbp_workspace_size() bytes, 256-byte
                                aligned; NULL = the library allocates it stream-ordered */
    size_t workspace_bytes;
    void* kernel_events[2];  /* optional cudaEvent_t pair, recorded on `stream` right before
                                and right after the schedule kernel (for timing it alone) */
    int32_t check_method;    /* gfbp_check_method for the horizontal pass (Eq. 3) */
    int32_t sus_width;       /* SUS, LANES layout: lane teams per frame, 1, 2, 4 or 8
                                (0 = chosen from the frame count).  Teams > 1 update
                                columns that share no check at the same time; every
                                column still sees the values of the sequential order,
                                so results are the same bit for bit. */
    int32_t layout;          /* gfbp_layout */
    int32_t sus_partials;    /* gfbp_sus_partials */
    int32_t* zero_sums;      /* device [F] or NULL: per frame, the number of message and
                                posterior normalisations (r_ij by Eq. 3, q_ij by Eq. 4, Q_j
                                by Eq. 5) whose sum was zero or not finite and that fell
                                back to the uniform vector, set by this call (a device-side
                                anomaly status word: decoding goes on, nothing traps).  A
                                zero sum arises where the evidence contradicts itself, e.g.
                                a symbol observed without erasure against a syndrome that
                                excludes it. */
} gfbp_options;

/*
 * Scratch bytes that gfbp_decode (step = 0) or gfbp_step (step = 1) needs for
 * n_frames frames with this schedule and prior.
 */
gfbp_status gfbp_workspace_size(const gfbp_code* code, int32_t n_frames, gfbp_schedule schedule,
                                const gfbp_prior* prior, int32_t step, size_t* bytes);

/*
 * Decode n_frames independent frames (Sec. 2).  Per frame: channel
 * likelihoods times the source prior give p_j; q_ij <- p_j; then iterations of
 * the schedule — PUS: every r_ij by Eq. 3 from the previous iteration's q,
 * then every q_ij and Q_j by Eqs. 4-5; SUS: for j = 0..N-1 in order, r_ij for
 * the checks of column j from the current q, then q_ij and Q_j of column j —
 * each followed by the hard decision (argmax of Q_j, lowest symbol on ties)
 * and the test H x = z; the frame stops at the first iteration that passes or
 * after max_iter.  With a Markov prior the block priors are re-estimated
 * (Eq. 6-7) from the finished iteration's Q and used in the next one.
 *   obs       device, see gfbp_channel_kind.
 *   max_iter  >= 1.
 *   x_hat     device [F][N]: decided symbols of the last iteration.
 *   iters     device [F]: iterations run (1..max_iter); -1 marks a frame whose
 *             decode gave up on an internal bounded wait (SUS with sus_width
 *             > 1 only; no such wait is expected to run out), its x_hat and
 *             converged flag are then not valid.
 *   converged device [F]: 1 when H x_hat = z.
 */
gfbp_status gfbp_decode(const gfbp_code* code, int32_t n_frames, const float* obs, gfbp_channel channel,
                        gfbp_schedule schedule, const gfbp_prior* prior, int32_t max_iter, uint8_t* x_hat,
                        int32_t* iters, uint8_t* converged, const gfbp_options* options, void* stream);

/*
 * gfbp_decode without any device allocation.  The paper has no counterpart;
 * this entry point exists for callers that cannot allocate device memory on
 * their decode path: real-time receivers that fix their device footprint at
 * start-up and forbid allocation per request (allocation time and
 * fragmentation are unpredictable), and plug-ins into programs whose own
 * caching allocator already holds the free device memory, where a cudaMalloc
 * of the library could fail or fragment that pool.
 *   Arguments, outputs and results are those of gfbp_decode.  The scratch is
 *   a static 32 MiB device array inside the library (reserved on every device
 *   that loads the library, until the process exits); options->workspace is
 *   ignored.  A batch whose scratch (gfbp_workspace_size) exceeds 32 MiB is
 *   rejected with GFBP_EINVAL before any launch; decode it in smaller calls.
 *   The first call on a device, with that device current, looks up the
 *   array's device address (cudaGetSymbolAddress); make that first call
 *   before any stream capture.
 *   All calls share the one array: calls whose work overlaps on the GPU (on
 *   different streams or host threads, without ordering between them) race
 *   and corrupt each other's results.  No device memory is allocated or freed.
 */
gfbp_status gfbp_decode_noalloc(const gfbp_code* code, int32_t n_frames, const float* obs, gfbp_channel channel,
                                gfbp_schedule schedule, const gfbp_prior* prior, int32_t max_iter, uint8_t* x_hat,
                                int32_t* iters, uint8_t* converged, const gfbp_options* options, void* stream);

/*
 * Exactly one iteration of the schedule from a caller-supplied state, for
 * lock-step comparison with a reference.
 *   msg        device [F][E][q] in/out: q_ij before the iteration; q_ij after it.
 *   prior_in   device [F][K][q]: block priors used in this iteration (Markov only).
 *   prior_out  device [F][K][q]: Eq. 6-7 from this iteration's Q (Markov only; may be NULL).
 *   post       device [F][N][q]: Q_j after the iteration.
 *   x_hat      device [F][N]; sat device [F]: 1 when H x_hat = z.
 * options->xhat_trace and no_early_stop are ignored.
 */
gfbp_status gfbp_step(const gfbp_code* code, int32_t n_frames, const float* obs, gfbp_channel channel,
                      gfbp_schedule schedule, const gfbp_prior* prior, float* msg, const float* prior_in,
                      float* prior_out, float* post, uint8_t* x_hat, uint8_t* sat,
                      const gfbp_options* options, void* stream);

/* ------------------------------------------------ Walsh-Hadamard transform */
/*
 * y[v] = WHT(x[v]) for n q-vectors: y[b] = sum_a (-1)^popcount(a AND b) x[a],
 * the transform behind the convolution theorem of Eq. 3 (unnormalised; apply
 * it twice and divide by q for the identity).  x, y: device [n][q] float32,
 * 16-byte aligned; y may equal x.
 *   GFBP_WHT_SIMT    FP32 butterflies on the CUDA cores (any q).
 *   GFBP_WHT_TENSOR  the +-1 Hadamard matrix as H_{q/16} (x) H_16: every
 *                    16-entry chunk contracted with H_16 on the tensor cores
 *                    (each x split into FP16 high and low parts, FP32
 *                    accumulation), then FP32 butterflies across the q/16
 *                    chunks; q in {16, ..., 256}.  Each vector is scaled by
 *                    a power of two to a largest |x| in [1, 2) first (undone
 *                    exactly).  Error per output below
 *                    2^-19 sum_a |x[a]| + q 2^-24 max_a |x[a]| (tested).
 * Enqueued on `stream`.
 */
typedef enum { GFBP_WHT_SIMT = 0, GFBP_WHT_TENSOR = 1 } gfbp_wht_method;
gfbp_status gfbp_wht(const float* x, float* y, int64_t n, int32_t q, int32_t method, void* stream);

/*
 * Self-test of the decoder kernels' bounded device waits: runs one of them on
 * a condition that never comes true, on `stream`, and waits for it.
 *   which 0: the mbarrier wait of the bulk copies (an mbarrier that expects
 *            one arrival; none is made).
 *   which 1: the watermark wait of the multi-team SUS kernel (a progress word
 *            that never passes the awaited column).
 *   completed  host: 1 if the wait completed, 0 if it ran out.
 * Returns GFBP_ETIMEOUT when the wait ran out, which is the expected outcome
 * (the kernel returns normally and the context stays usable); GFBP_OK would
 * mean the wait completed without its condition.  Takes up to about a second.
 */
gfbp_status gfbp_wait_selftest(int32_t which, int32_t* completed, void* stream);

/* --------------------------------------------------------------- batching */
/*
 * Frames of several codes — uneven q and N — decoded by one persistent launch
 * over a device frame table (the decoding of every frame is that of
 * gfbp_decode, Sec. 2).  gfbp_batch_create validates the items, allocates one
 * device block (frame table, per-item workspaces) and copies the item
 * descriptors, synchronously; gfbp_batch_run then only enqueues kernels on
 * `stream` (no allocation, no host synchronisation, no host-to-device copy),
 * so a run can be captured in a CUDA graph and replayed.  Each run re-reads
 * the items' obs and rewrites their outputs; runs of one batch must not
 * overlap on the GPU (they share the workspaces).
 * Limits: 1..65536 items; every code with row degree <= 6 and column degree <= 3;
 * codes of one field size must share the field polynomial.
 */
typedef struct {
    const gfbp_code* code;
    int32_t n_frames;
    const float* obs;          /* device, as for gfbp_decode */
    gfbp_channel channel;
    const gfbp_prior* prior;   /* NULL = i.i.d.; read during gfbp_batch_create only */
    uint8_t* x_hat;            /* device [F][N] */
    int32_t* iters;            /* device [F] */
    uint8_t* converged;        /* device [F] */
} gfbp_batch_item;

typedef struct gfbp_batch gfbp_batch;

/* options: only check_method AUTO is used; per-call options are rejected. */
gfbp_status gfbp_batch_create(const gfbp_batch_item* items, int32_t n_items, gfbp_schedule schedule,
                              int32_t max_iter, const gfbp_options* options, gfbp_batch** out);
gfbp_status gfbp_batch_run(gfbp_batch* batch, void* stream);
/* Kernel variant chosen for every item (host [n_items]; values as in gfbp_autotune). */
gfbp_status gfbp_batch_variants(const gfbp_batch* batch, int32_t* variants);
/* Pin the kernel variant of every item (host [n_items], values as in
 * gfbp_autotune); each must be one that gfbp_autotune may choose for the
 * item's q and the batch's schedule (GFBP_EINVAL otherwise, nothing changed).
 * Synchronous; not during a run of the batch. */
gfbp_status gfbp_batch_set_variants(gfbp_batch* batch, const int32_t* variants);
void gfbp_batch_destroy(gfbp_batch* batch);

/*
 * Autotuner: time every kernel variant that computes the same check-node
 * route for this code and schedule (SUS: the level schedule with a CTA per
 * frame, the team kernel with a warp per frame (q = 4, 8, 16), the group
 * kernel with a lane group per frame) on the caller's sample of n_frames
 * frames, and remember the fastest for codes of the same (q, N, M, E) and
 * schedule on this device; later gfbp_batch_create calls use it.
 * Synchronous; allocates its own scratch.  *chosen receives the variant:
 * 0-2 team q = 4/8/16, 3-6 group probability route q = 2/4/8/16,
 * 7-10 group transform route q = 32/64/128/256, 11-14 levels probability
 * route q = 2/4/8/16, 15-18 levels transform route q = 32/64/128/256,
 * 19-23 levels TENSOR route q = 16/32/64/128/256, 24-27 levels probability
 * route by lane groups q = 32/64/128/256.  Items decode by AUTO's route (the
 * default without tuning: 11-14, 24-25 and 17-18), so this chooses among its
 * variants only; PUS has one variant per q.  The variants of the other
 * routes (7-8 and 15-16, 26-27, 19-23) are explicit choices for
 * gfbp_batch_set_variants.
 */
gfbp_status gfbp_autotune(const gfbp_code* code, int32_t n_frames, const float* obs, gfbp_channel channel,
                          gfbp_schedule schedule, const gfbp_prior* prior, int32_t max_iter, void* stream,
                          int32_t* chosen);

/* ---------------------------------------------------------------- serving */
/*
 * Continuous batching of decode requests (each the decoding of gfbp_decode,
 * Sec. 2).  The server reserves one device pool of hbm_budget_bytes and runs
 * a worker thread in rounds: queued requests are admitted in arrival order
 * while their device footprint (message workspace, inputs, outputs, state)
 * fits in the pool's free space; one persistent launch per schedule then
 * advances every frame of every resident request by at most round_iters
 * iterations from where it stopped (message state stays resident between
 * rounds); frames that stopped are retired after the round, their outputs
 * written to the request's host buffers and their space freed.  Requests that
 * arrive while others are on the GPU join at the next round boundary.  A
 * frame's result does not depend on what else is resident.
 * Codes: row degree <= 6, column degree <= 3; codes of one field size must
 * share the field polynomial.
 */
typedef struct gfbp_server gfbp_server;

typedef struct {
    const gfbp_code* code;
    int32_t n_frames;
    const float* obs;          /* HOST [F][N][p] (or [F][N][q] log-likelihoods); copied at submit */
    gfbp_channel channel;      /* frame_param, if set, is a HOST [F] array, copied at submit */
    const gfbp_prior* prior;   /* NULL = i.i.d.; copied at submit */
    gfbp_schedule schedule;
    int32_t max_iter;
    uint8_t* x_hat;            /* HOST [F][N], written before the request completes */
    int32_t* iters;            /* HOST [F] */
    uint8_t* converged;        /* HOST [F] */
} gfbp_request;

typedef struct {
    double latency_us;         /* submit to outputs written */
    double queue_us;           /* submit to admission */
    int32_t rounds;            /* rounds the request was resident */
} gfbp_result;

typedef struct {
    int32_t queued, resident, peak_resident;
    int64_t rounds, completed;
    size_t bytes_in_use, peak_bytes;
} gfbp_server_stats_t;

/* round_iters >= 1: iterations a resident frame advances per round at most.
 * Requests whose iteration costs at least eight GF(16), N = 1000 frame
 * iterations run in a lane of rounds of their own, on their own stream, that
 * light requests never wait for; in the light lane a frame costing more than
 * one such unit advances proportionally fewer iterations per round (at
 * least one). */
gfbp_status gfbp_server_create(size_t hbm_budget_bytes, int32_t round_iters, gfbp_server** out);
/* Queue a request (thread-safe).  GFBP_EINVAL if its footprint exceeds the
 * whole budget; GFBP_EBUSY while the server drains.  The output buffers must
 * stay valid until gfbp_server_wait returns for this id. */
gfbp_status gfbp_server_submit(gfbp_server* server, const gfbp_request* request, uint64_t* id);
/* Wait at most timeout_us for request id (GFBP_ETIMEOUT otherwise; the request
 * stays queued or resident and can be waited for again).  On success the id is
 * released. */
gfbp_status gfbp_server_wait(gfbp_server* server, uint64_t id, int64_t timeout_us, gfbp_result* result);
gfbp_status gfbp_server_stats(gfbp_server* server, gfbp_server_stats_t* stats);
/* Refuse new requests and return once every queued and resident one is done. */
gfbp_status gfbp_server_drain(gfbp_server* server);
/* Finish the admitted and queued work, stop the worker and free the pool. */
void gfbp_server_destroy(gfbp_server* server);

#ifdef __cplusplus
}
#endif

#endif /* GFBP_H */
