/*
 * krux.h -- C ABI of the GB300 (sm_103a) Kruskal-Wallis SNP x trait scan.
 *
 * The library computes, for every pair of an expression trait n and a genetic
 * marker (SNP) m, the tie-corrected Kruskal-Wallis statistic H and its
 * chi-square p-value, and returns the pairs with p < P_c (Qi et al., "kruX:
 * Matrix-based non-parametric eQTL discovery", arXiv:1307.3519).  Notation:
 * T traits, S SNPs, N samples (the paper's N, M, K).
 *
 * Conventions shared by every entry point:
 *  - Pointers named "device" are CUDA device pointers owned by the caller; the
 *    library never frees them.  Pointers named "host" are ordinary host memory.
 *  - The context owns its workspace and the rank sets it creates.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Work is enqueued on it; calls that return counts (n_hits)
 *    synchronise that stream before returning.
 *  - Every call returns a krux_status; nothing throws across the ABI.  After a
 *    failure krux_last_error(ctx) holds a one-line message.  A failure leaves
 *    the caller's output buffers unspecified.
 *  - One context per host thread; calls on one context are not re-entrant.
 */
#ifndef KRUX_H
#define KRUX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  KRUX_OK = 0,
  KRUX_EINVAL = 1,        /* bad argument or input value (e.g. genotype code outside {-1,0,1,2}) */
  KRUX_ENOMEM = 2,        /* device or host allocation failed */
  KRUX_ECUDA = 3,         /* a CUDA runtime / driver call failed */
  KRUX_EOVERFLOW = 4,     /* more hits than hit_capacity: n_hits holds the exact total */
  KRUX_ETIMEOUT = 5,      /* a bounded device-side wait gave up; outputs are invalid */
  KRUX_EUNSUPPORTED = 6   /* valid request this build cannot serve (e.g. no sm_103a device) */
} krux_status;

typedef struct krux_ctx krux_ctx;
typedef struct krux_rankset krux_rankset;

/* One significant pair.  d0, d1 are the exact centred rank sums
 * D_i = 2*S_i - N_i*(K+1) of genotype groups 0 and 1 (S_i of Eq. 4; D_2 = -D_0 - D_1).
 * The FP64 statistic and p-value of hit j are written to hit_H[j], hit_p[j]. */
typedef struct {
  uint32_t trait;
  uint32_t snp;
  int32_t d0;
  int32_t d1;
} krux_hit;

/* krux_opts.flags bits.
 * KRUX_FLAG_MULTIALLELIC: genotype codes 0..4 (section "Input data": markers take
 *   values 0..l with any number of alleles, also varying between markers; here
 *   l <= 4, so up to five genotype groups and df up to 4; the chi-square tail of
 *   df 3 and 4 is computed in closed form).  Without it codes must be in
 *   {-1, 0, 1, 2}.  The flag works with krux_scan, krux_scan_cis,
 *   krux_scan_grouped and their graphs, on complete expression (no NaN) without
 *   dense output; permutation batches and the plain form take biallelic markers
 *   only (KRUX_EUNSUPPORTED).  Biallelic data scanned with the flag give the same
 *   hits, H and p. */
#define KRUX_FLAG_MULTIALLELIC 1

/* Scan options (section "P-value calculation and empirical FDR correction": the
 * threshold P_c; section "Data slicing": a slice of markers starting at a given
 * marker). */
typedef struct {
  double pthresh;          /* P_c, 0 < P_c < 1: a pair is a hit iff p < P_c */
  int64_t hit_capacity;    /* entries available in hits / hit_H / hit_p */
  int64_t snp_begin;       /* scan SNP rows [snp_begin, snp_end) of the genotype matrix */
  int64_t snp_end;         /* snp_end <= 0 means S */
  double *dense_H;         /* optional device [T][snp_end-snp_begin] FP64 H of every pair, NULL = off */
  double *dense_p;         /* optional device, same layout, FP64 p of every pair */
  double recheck_margin;   /* relative band around the threshold decided in FP64; <= 0 -> 1e-4 */
  int32_t flags;           /* KRUX_FLAG_* bits, 0 = none */
  int32_t reserved_;
} krux_opts;

/* Per-call kernel timings (CUDA events on the call's stream) when profiling is on. */
typedef struct {
  float ms_rank;        /* rank transform (krux_rank) */
  float ms_pack;        /* genotype packing */
  float ms_scan;        /* fused tcgen05 scan kernel alone, or plain GEMM + epilogue */
  float ms_finalize;    /* FP64 H / p of the hit list */
  float ms_gemm;        /* plain form: library GEMM part of ms_scan */
  int32_t launches;     /* kernels the last call launched */
  int32_t scan_grid;    /* CTAs of the fused scan launch */
  int64_t pairs;        /* SNP x trait pairs the last call tested */
  int32_t scan_form;    /* kernel form of the fused scan launch: 0 plain, 1 markers with up to
                           five groups, 2 permutation batch, 3 general (dense, cis, NaN
                           beyond the plain form's coefficient sets), 4 plain permutation
                           batch, 5 plain with NaN expression */
  int32_t reserved_;
} krux_profile;

/* Create a context on CUDA device `device` (must be sm_103 for the fused path).
 * *ctx receives the handle. */
krux_status krux_create(krux_ctx **ctx, int device);
void krux_destroy(krux_ctx *ctx);
const char *krux_status_string(krux_status s);
const char *krux_last_error(const krux_ctx *ctx);

/* Rank transform (section "Input data": ranks per trait row; section "Handling
 * missing values": NaN samples are left out and get 0; section "Handling tied
 * data": ties get the average rank and the factor sum(t^3 - t) is computed while
 * ranking).
 *   expr : device float32 [T][ld] row-major, NaN = missing; 1 <= N <= 512, ld >= N.
 *   *out : receives a rank set owned by ctx (free with krux_rankset_free).
 * Stores, per trait, the centred ranks 2*rank - (K+1), the tie sum and K. */
krux_status krux_rank(krux_ctx *ctx, const float *expr, int T, int N, int64_t ld,
                      krux_rankset **out, void *stream);
void krux_rankset_free(krux_ctx *ctx, krux_rankset *rs);
/* Copies a rank set out: centred: device int16 [T][N] (2*rank - (K+1), 0 at NaN);
 * tie: device int64 [T] (sum of t^3 - t); K: device int32 [T].  Any may be NULL. */
krux_status krux_rankset_export(krux_ctx *ctx, const krux_rankset *rs, int16_t *centred,
                                int64_t *tie, int32_t *K, void *stream);

/* Fused scan (Eq. 4 rank sums by tensor-core contraction, Eq. 2 statistic with
 * the tie factor, chi-square tail, threshold, hit list).
 *   geno : device int8 [S][ldg] row-major, codes 0/1/2, -1 = missing; any other
 *          code -> KRUX_EINVAL.  Same sample order and N as the rank set.
 *   hits, hit_H, hit_p : device outputs of opts->hit_capacity entries, in
 *          unspecified order; hits must be 16-byte aligned (else KRUX_EINVAL).
 *          SNP indices are rows of geno (slice offsets included).  Which pairs
 *          are hits is decided with the FP64 chi-square tail (p < pthresh); H is
 *          computed in FP64 from the exact rank sums; the reported p of df 1 and 2
 *          comes from an FP64 range reduction with FP32 exp2 / erfcx parts
 *          (relative error a few 1e-7, always below pthresh for a hit).
 *   n_hits : host; receives the exact number of hits, also when it exceeds the
 *          capacity (then the first hit_capacity found are stored and the call
 *          returns KRUX_EOVERFLOW).
 * SNPs with missing genotypes are grouped by missing-sample pattern and scanned
 * against ranks recomputed over the samples they have (section "Handling
 * missing values"). */
krux_status krux_scan(krux_ctx *ctx, const krux_rankset *rs, const int8_t *geno, int64_t S,
                      int64_t ldg, const krux_opts *opts, krux_hit *hits, double *hit_H,
                      double *hit_p, int64_t *n_hits, void *stream);

/* End-to-end scan from host memory (the paper's whole analysis of section
 * "Implementation": input matrices in, significant pairs out): copies the
 * inputs to the device, runs krux_rank and krux_scan there, and copies the hit
 * list back.
 *   expr : HOST float32 [T][lde], as krux_rank (NaN = missing).
 *   geno : HOST int8 [S][ldg], as krux_scan.
 *   hits, hit_H, hit_p : HOST outputs of opts->hit_capacity entries; *n_hits as
 *          in krux_scan (exact count; KRUX_EOVERFLOW when above the capacity,
 *          with the first hit_capacity records copied).
 * Page-locked host buffers (cudaHostAlloc or cudaHostRegister) copy at the
 * link's rate; pageable ones work but copy through a bounce buffer.  Each input
 * is one cudaMemcpyAsync (cudaMemcpy2DAsync when its leading dimension exceeds
 * N) into device memory the context keeps between calls; the genotypes' copy runs
 * on a stream the context owns, beside the rank transform on `stream`.  Outputs in page-locked
 * memory mapped into the device's address space (cudaHostAlloc, or
 * cudaHostRegister with cudaHostRegisterMapped; `hits` 16-byte aligned) are
 * written by the library's kernels directly; other outputs are filled by three
 * copies of min(*n_hits, capacity) records from a device list.  opts->dense_H / dense_p must be
 * NULL (dense output is a device-side option of krux_scan).  The call
 * synchronises `stream` before returning. */
krux_status krux_scan_host(krux_ctx *ctx, const float *expr, int T, int N, int64_t lde,
                           const int8_t *geno, int64_t S, int64_t ldg, const krux_opts *opts,
                           krux_hit *hits, double *hit_H, double *hit_p, int64_t *n_hits,
                           void *stream);

/* Plain two-pass form of the same scan, kept as the measured comparison point:
 * a library FP16 GEMM writes the T x 2S rank-sum matrix (in SNP slices) to device
 * memory, then a separate epilogue kernel reads it back.  Same arguments and
 * results as krux_scan (complete genotypes only: -1 codes -> KRUX_EUNSUPPORTED). */
krux_status krux_scan_plain(krux_ctx *ctx, const krux_rankset *rs, const int8_t *geno,
                            int64_t S, int64_t ldg, const krux_opts *opts, krux_hit *hits,
                            double *hit_H, double *hit_p, int64_t *n_hits, void *stream);

/* Permutation null (section "P-value calculation and empirical FDR correction":
 * the scan repeated, with the same P_c, with the columns of the expression ranks
 * permuted).
 *   perms : device int32 [P][N], each row a permutation of 0..N-1; sample k of
 *           permutation q takes the expression of sample perms[q][k].
 *   minp  : device double [P][T]: per permutation and trait, the minimum p over
 *           the scanned SNPs.
 *   fdr_hist : optional device uint64 [1 + P][fdr_bins] (NULL = off), zeroed and
 *           filled by the call: row 0 counts the real data's stored hits, row q the
 *           pairs of permutation q with p' < P_c, both by bin
 *           b = floor((-log10 p - (-log10 P_c)) / fdr_bin_width), clamped to
 *           [0, fdr_bins).  Summing bins b.. gives the count of pairs with
 *           p <= P_c * 10^(-b * fdr_bin_width), from which the empirical FDR of
 *           that threshold is the mean permuted count over the real count.
 *           fdr_bins >= 1 and fdr_bin_width > 0 when fdr_hist is given.  Row 0 is
 *           complete only when the hits fit the capacity (else KRUX_EOVERFLOW).
 * The unpermuted scan's hits are returned as in krux_scan.  With more than 65,536
 * SNPs a short seed pass over the first 16,384 runs first and primes the minimum-p
 * search with lower bounds; both launches are enqueued back to back on `stream`
 * (the rows of perms are checked on the host first, the hit counts read back at
 * the end), and krux_graph_permute captures the same two launches. */
krux_status krux_permute(krux_ctx *ctx, const krux_rankset *rs, const int8_t *geno, int64_t S,
                         int64_t ldg, const int32_t *perms, int P, const krux_opts *opts,
                         double *minp, krux_hit *hits, double *hit_H, double *hit_p,
                         int64_t *n_hits, uint64_t *fdr_hist, int fdr_bins,
                         double fdr_bin_width, void *stream);

/* cis scan (the paper's cis-eQTL analysis keeps marker-trait pairs within 1 Mbp
 * of each other): as krux_scan, but only pairs with
 * |snp_pos[snp] - trait_pos[trait]| <= window are tested and reported, and the
 * work is pruned to them: every SNP tile meets only the trait tiles its window
 * reaches.
 *   snp_pos   : device int64 [S], a global coordinate per SNP row (for several
 *               chromosomes, e.g. chromosome * 2^40 + base position), nondecreasing;
 *   trait_pos : device int64 [T], the coordinate of each trait's gene, same scale,
 *               nondecreasing (sort the traits before ranking);
 *   window    : >= 0, same units.
 * Unsorted coordinates, window < 0 or dense output -> KRUX_EINVAL. */
krux_status krux_scan_cis(krux_ctx *ctx, const krux_rankset *rs, const int8_t *geno, int64_t S,
                          int64_t ldg, const int64_t *snp_pos, const int64_t *trait_pos,
                          int64_t window, const krux_opts *opts, krux_hit *hits, double *hit_H,
                          double *hit_p, int64_t *n_hits, void *stream);

/* Parametric statistics on the same tiles (the paper compares kruX with the
 * linear and ANOVA models of matrix-eQTL on the same data): the contraction of
 * the scan with the centred ranks replaced by standardised values
 * (x - mean) / sd per trait, then
 *   model 0: one-way ANOVA over the genotype groups, F with (groups - 1,
 *            N - groups) df, p = upper F tail;
 *   model 1: least-squares regression on the dosage (the code 0/1/2), t with
 *            N - 2 df, p = two-sided t tail.
 * The fused test runs on FP16 values with a wide band; every pair in it is
 * recomputed in FP64 from `expr` and kept iff p < P_c, so the hit set and the
 * FP64 statistic and p are those of the definitions.
 *   expr : device float32 [T][ld], no NaN (-> KRUX_EINVAL); 4 <= N <= 512.
 *   geno : device int8 [S][ldg], codes 0, 1, 2 (a -1 -> KRUX_EUNSUPPORTED).
 *   hits : records with d0 = d1 = 0; hit_stat receives F (model 0) or t
 *          (model 1), hit_p its p-value; 16-byte aligned hits as in krux_scan.
 * opts: pthresh, hit_capacity and the SNP slice are used; flags must be 0 and
 * dense output is not available.  n_hits is exact; if the band's work list
 * (hit_capacity + 2^20 entries) overflows the call returns KRUX_EOVERFLOW with
 * n_hits an upper bound. */
krux_status krux_scan_parametric(krux_ctx *ctx, const float *expr, int T, int N, int64_t ld,
                                 const int8_t *geno, int64_t S, int64_t ldg, int model,
                                 const krux_opts *opts, krux_hit *hits, double *hit_stat,
                                 double *hit_p, int64_t *n_hits, void *stream);

/* Test hook (host only): the FP64 tails the parametric finalisation uses.
 * kind 0: P(F(d1, d2) > x); kind 1: P(|T(d1)| > x); kind 2: I_x(d1, d2). */
double krux_debug_tail(int kind, double x, double d1, double d2);

/* One cohort of a grouped scan: its own rank set (any N <= 512), genotypes and
 * hit outputs; n_hits is written by krux_scan_grouped. */
typedef struct {
  const krux_rankset *rs;
  const int8_t *geno;     /* device int8 [S][ldg] */
  int64_t S;
  int64_t ldg;
  krux_hit *hits;         /* device, hit_capacity entries */
  double *hit_H;
  double *hit_p;
  int64_t hit_capacity;
  int64_t n_hits;         /* out */
} krux_cohort;

/* Several cohorts of uneven sample counts in one persistent launch.  opts gives
 * the threshold (its hit_capacity and slice fields are ignored).  Returns
 * KRUX_EOVERFLOW if any cohort overflowed. */
krux_status krux_scan_grouped(krux_ctx *ctx, krux_cohort *cohorts, int n_cohorts,
                              const krux_opts *opts, void *stream);

/* P permutations of 0..N-1 into host int32 [P][N]: permutation q is a
 * Fisher-Yates shuffle (i = N-1 .. 1, j = x mod (i+1), swap) driven by SplitMix64
 * started at state seed + q. */
krux_status krux_make_perms(uint64_t seed, int P, int N, int32_t *out);

/* Record per-kernel CUDA-event timings of each call (adds event overhead). */
krux_status krux_set_profiling(krux_ctx *ctx, int enable);
krux_status krux_get_profile(const krux_ctx *ctx, krux_profile *out);

/* Fused scan for callers that cannot allocate device memory (no paper
 * counterpart: this is a deployment variant of krux_scan).  Code running under
 * an allocator that owns the whole device, plugins inside such processes, and
 * latency-critical paths where an allocation may block or fail can call this
 * instead: it needs no context and calls no cudaMalloc, cudaFree or allocating
 * library routine.  All scratch memory comes from one fixed 16 MiB device array
 * inside the library, which every GPU that loads the library keeps until the
 * process exits.
 *   expr, T, N, ld, geno, S, ldg, pthresh : as krux_rank / krux_scan, with
 *          T <= 4096, N <= 256 and complete genotypes (a -1 code returns
 *          KRUX_EUNSUPPORTED); any S (SNPs are processed in slices of 4096).
 *   hits, hit_H, hit_p : device outputs of hit_capacity entries.  At most
 *          262,144 hits are stored per call; *n_hits (host) is always the exact
 *          count, and KRUX_EOVERFLOW is returned when it exceeds what was stored.
 * Sizes beyond these limits return KRUX_EINVAL before any device work.  The
 * first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current, so make it before any stream
 * capture.  Every call on a device shares the array, and the previous call's
 * contents stay in it (each call clears what must start at zero); calls that
 * overlap on the GPU race, so issue them on one stream or serialise them.  The
 * call synchronises `stream` before returning.  Its kernels give up a spinning
 * wait after a fixed limit of 4x10^9 SM cycles (about two seconds) and then
 * return KRUX_ETIMEOUT; krux_set_wait_limit, which sets a context's limit, has
 * no effect here (this entry point has no context). */
krux_status krux_scan_noalloc(const float *expr, int T, int N, int64_t ld, const int8_t *geno,
                              int64_t S, int64_t ldg, double pthresh, krux_hit *hits,
                              double *hit_H, double *hit_p, int64_t hit_capacity,
                              int64_t *n_hits, void *stream);

/* Tile-shape control for the autotuner and tests: layout 0 = 128-byte swizzled
 * K atoms of 64 samples, 1 = 32-byte swizzled atoms of 16 samples, -1 = automatic;
 * nc = SNP chunks (64 SNPs each) kept resident, nA = rank-tile pipeline stages,
 * ka = samples per rank stage (a multiple of 64; 0 = the whole K); nc = nA = 0
 * (and ka = 0) = automatic.  A shape that does not fit shared memory makes the
 * next scan return KRUX_EINVAL. */
krux_status krux_set_tuning(krux_ctx *ctx, int layout, int nc, int nA, int ka);

/* Autotuner (the tile shape is the project's own choice per sample width; the
 * paper has no counterpart).  Times the fused scan of `rs` against the first
 * min(S, 65536) SNPs of `geno` (device int8 [S][ldg]) at threshold pthresh for
 * every launch shape that fits shared memory (both swizzle layouts, 1-4
 * resident chunks, 2-4 rank stages, whole-K or 64-sample K blocks, and the
 * automatic choice), three runs each, and keeps the fastest for the rank set's
 * padded width Np: later scans whose widest group has that width use it, unless
 * krux_set_tuning sets a shape.  shape_out (host int32[4], may be NULL) receives
 * {layout, nc, nA, ka} of the winner (-1/0 entries = automatic).  Uses a
 * temporary 40 MB device buffer; synchronises `stream`. */
krux_status krux_autotune(krux_ctx *ctx, const krux_rankset *rs, const int8_t *geno, int64_t S,
                          int64_t ldg, double pthresh, void *stream, int32_t *shape_out);

/* CUDA graphs (the batched launch captured once and replayed; the paper has no
 * counterpart).  krux_graph_scan / krux_graph_permute / krux_graph_grouped take
 * the arguments of krux_scan / krux_permute / krux_scan_grouped (without
 * n_hits and stream), plan the call once (the SNP groups, the launch shape, the
 * work items) and capture its device work in a graph: for permutations the row
 * gathers, then the packing of every group, the fused scan, the hit
 * compaction, the FP64 finalisation (its hit count read on the device), the
 * min-p conversion and the read-back of the hit counts into pinned host
 * memory.  A replay (krux_graph_launch) reads the current contents of every
 * buffer given at capture: new genotypes, ranks or permutations of the same
 * shapes are scanned without any host work.  The graph owns a private
 * workspace; the rank sets and all caller buffers must outlive it.
 * Restrictions: complete genotypes at capture (a -1 code -> KRUX_EUNSUPPORTED);
 * a -1 that appears in a replay is left out of the scan and reported by
 * krux_graph_wait as KRUX_EUNSUPPORTED; a replayed permutation entry outside
 * 0..N-1 reads as zeros and is reported as KRUX_EINVAL (replays check only the
 * range of entries, not that a row is a permutation).
 * *out receives the graph (free with krux_graph_destroy). */
typedef struct krux_graph krux_graph;
krux_status krux_graph_scan(krux_ctx *ctx, const krux_rankset *rs, const int8_t *geno, int64_t S,
                            int64_t ldg, const krux_opts *opts, krux_hit *hits, double *hit_H,
                            double *hit_p, krux_graph **out);
krux_status krux_graph_permute(krux_ctx *ctx, const krux_rankset *rs, const int8_t *geno,
                               int64_t S, int64_t ldg, const int32_t *perms, int P,
                               const krux_opts *opts, double *minp, krux_hit *hits,
                               double *hit_H, double *hit_p, uint64_t *fdr_hist, int fdr_bins,
                               double fdr_bin_width, krux_graph **out);
krux_status krux_graph_grouped(krux_ctx *ctx, const krux_cohort *cohorts, int n_cohorts,
                               const krux_opts *opts, krux_graph **out);
/* Enqueues one replay on `stream` (asynchronous). */
krux_status krux_graph_launch(krux_graph *g, void *stream);
/* Waits for the last replay and writes the exact hit count of each of its
 * n_lists >= (number of hit lists: 1, or the cohort count) lists to n_hits
 * (host).  Returns KRUX_OK, KRUX_EOVERFLOW (some list's count exceeds its
 * capacity; the first `capacity` hits are stored), or a device-side error. */
krux_status krux_graph_wait(krux_graph *g, int64_t *n_hits, int n_lists);
const char *krux_graph_last_error(const krux_graph *g);
void krux_graph_destroy(krux_graph *g);

/* Test hook (no GPU needed): the pipeline shape a scan of one group of N samples
 * would use, after the same shared-memory plan check every launch passes.
 * with_nan: 0 complete data, 1 NaN expression in the general form (2-bit codes),
 * 2 the plain form on complete data (with its hit-event ring), 3 the plain form's
 * NaN variant (coefficient sets).  out[7] = {samples per rank stage, rank stages,
 * B region bytes, resident chunks, K blocks per step, B chunk stride,
 * shared-memory bytes}.  Returns KRUX_OK, KRUX_EUNSUPPORTED if no sound plan of
 * that kind exists, KRUX_EINVAL for arguments out of range. */
krux_status krux_debug_plan(int N, int with_nan, int layout, int nc, int nA, int ka, int32_t *out);

/* Test hook: device-side waits give up after `cycles` SM clock cycles (0 = the
 * default of about two seconds). */
krux_status krux_set_wait_limit(krux_ctx *ctx, long long cycles);

#ifdef __cplusplus
}
#endif

#endif /* KRUX_H */
