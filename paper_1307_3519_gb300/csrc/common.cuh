// common.cuh -- device-side data layouts shared by the kernels of the Kruskal-Wallis
// scan library (rank transform, genotype packing, fused tcgen05 scan, FP64
// finalisation, plain GEMM form) and by the host orchestration in abi.cu.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/krux.h"

namespace krux {

// ---- fixed tile geometry ---------------------------------------------------
constexpr int kTileM = 128;        // traits per MMA tile = TMEM lanes
constexpr int kChunkSnps = 64;     // SNPs per chunk
constexpr int kChunkRows = 128;    // B rows per chunk: [I_0 of 64 SNPs | I_1 of 64 SNPs]
constexpr int kMaxN = 512;         // samples: centred 2*rank fits FP16 exactly below 2048
constexpr int kAtomK = 64;         // K elements per 128-byte swizzle atom (fp16)
constexpr int kTmemSlots = 4;      // accumulator ring: 4 x 128 fp32 columns = all of TMEM
constexpr int kEpiWarps = 16;      // epilogue warps: 4 per TMEM lane quarter
constexpr int kEpiSnps = 16;       // SNPs of a chunk each epilogue warp evaluates
constexpr int kProducerWarp = 16;  // TMA producer
constexpr int kMmaWarp = 17;       // tcgen05.mma issuer, owns the TMEM allocation
constexpr int kScanThreads = 576;
// The plain scan form (complete data, chunks paired into N = 256 MMAs): each of
// its epilogue warps owns kFastSnps SNPs of one chunk of every accumulator pair
// for one TMEM lane quarter (32 traits); after them come the producer, the MMA
// issuer and two idle warps that complete their warpgroup, whose registers go to
// the epilogue warps (setmaxnreg: both splits use all registers of the launch).
constexpr int kFastSnps = 32;
constexpr int kFastEpiWarps = 4 * (2 * kChunkSnps / kFastSnps);  // 16
constexpr int kFastThreads = 32 * (kFastEpiWarps + 4);
// the register file is split among the 4 schedulers: at most 16384 per scheduler
constexpr int kFastRegsLaunch = (16384 / (32 * (kFastThreads / 128))) / 8 * 8;
constexpr int kFastRegsLow = 56;
constexpr int kFastRegsHigh =
    (kFastRegsLaunch + 4 * (kFastRegsLaunch - kFastRegsLow) / kFastEpiWarps) / 8 * 8;
static_assert(kFastEpiWarps == 16, "16 epilogue warps in the plain scan form");
static_assert(kFastThreads * kFastRegsLaunch <= 65536, "launch registers");
static_assert(4 * (kFastRegsLaunch - kFastRegsLow) >= kFastEpiWarps * (kFastRegsHigh - kFastRegsLaunch),
              "the epilogue's extra registers must come from the producer warpgroup");


// Hit events of the plain scan form are handed to the two idle warps of the
// producer warpgroup through a ring of shared-memory entries: an epilogue warp
// whose half-block (kEvSnps SNPs x 32 traits) has a candidate writes, for each
// trait lane that found one, an entry with that trait's kEvSnps centred sums and
// constants and the SNPs' metadata, and goes on; an event warp classifies the
// entry's pairs (FP64 inside the band) and appends the hit records.
constexpr int kEvSnps = kFastSnps / 2;  // 16
constexpr int kEvEntries = 32;
// A permuted pair the event warps passed on for its FP64 -ln p, decided after the
// launch: exact centred sums, group sizes, trait, and rank-matrix group | FDR-band
// flag << 16.
struct MinpPair {
  int32_t u, v;
  uint32_t n01, n2df;
  int32_t trait;
  int32_t agb;
};
static_assert(sizeof(MinpPair) == 24, "MinpPair is 24 bytes");

struct EvEntry {
  float u[kEvSnps], v[kEvSnps];                 // D_0, D_1 of SNP j for this trait
  float alpha[kEvSnps], beta[kEvSnps], gamma[kEvSnps];  // the SNPs' fast-test coefficients
  int32_t snp[kEvSnps];                         // output SNP index
  uint32_t n01[kEvSnps];                        // N_0 | N_1 << 16
  uint32_t n2df[kEvSnps];                       // N_2 | df << 16
  double cfac;                                  // 3 / (K(K+1)C) of the trait
  float tau;                                    // its fast-test bound
  int32_t trait;                                // its trait row
  int32_t group;
  int32_t ag;                                   // rank-matrix group (> 0: a permutation)
  float b1, b2;                                 // permutation: the classes' largest decided values
  uint32_t id1, id2;                            // and the identities of the pairs that have them
  int32_t nan;                                  // plain form with NaN: the trait's NaN samples
  int32_t pad_;
};
static_assert(sizeof(EvEntry) % 16 == 0, "event entries keep 16-byte alignment");
// shared memory of the ring: alignment slack, entries, a full barrier and a
// release count per entry, one 64-bit word (tickets claimed in the low 40 bits,
// epilogue warps done above)
constexpr size_t kEvRegion = 128 + kEvEntries * sizeof(EvEntry) + kEvEntries * 8 + kEvEntries * 4 + 8;
// Per-step trait constants staged in shared memory by the producer (one entry per
// 128-trait tile step): tau f32 [128] @0, 3/(K(K+1)C) f64 [128] @512, starting
// -ln p key f64 [128] @1536 (permutation batches), NaN count u16 [128] @2560; the
// two-sided plain form stages instead the classes' decided values with their pair
// identities, u64 [128][2] @1536 (it has no NaN).
constexpr int kTcDepth = 4;
constexpr int kTcBytes = 3584;

// ---- per-chunk SNP metadata (one 1536-byte blob per chunk of 64 SNPs) ------
// Fast-test coefficients: with u = D_0, v = D_1 (D_2 = -u - v) the statistic's
// quadratic form sum_i D_i^2 / N_i equals alpha (u + beta v)^2 + gamma v^2; alpha
// and gamma are pre-divided by the chi-square threshold h_df of the SNP's df so
// that one per-trait bound decides the test.
struct ChunkMeta {
  float alpha[kChunkSnps];      // (r0 + r2) / h_df
  float beta[kChunkSnps];       // r2 / (r0 + r2)
  float gamma[kChunkSnps];      // (r1 + r2 r0 / (r0 + r2)) / h_df
  int32_t snp[kChunkSnps];      // output SNP index, -1 = padding
  uint16_t n[3][kChunkSnps];    // genotype group sizes over non-missing samples
  uint8_t df[kChunkSnps];       // non-empty groups - 1
  uint8_t pad_[64];
};
static_assert(sizeof(ChunkMeta) == 1536, "ChunkMeta must be 1536 bytes");

// ---- markers with up to five genotype groups (section "Input data": values
// 0..l, any number of alleles, also varying between markers) ------------------
// A chunk holds 32 SNPs: rows [32i, 32i + 32) = I_i (i = 0..3) of SNPs 32c ..
// 32c + 31; group 4 is implicit (D_4 = -(D_0 + D_1 + D_2 + D_3), because the
// centred ranks of the present samples sum to zero).
constexpr int kMaxCodeM = 4;      // largest genotype code
constexpr int kChunkSnpsM = 32;   // SNPs per chunk
constexpr int kEpiSnpsM = 8;      // SNPs of a chunk each epilogue warp evaluates
struct ChunkMetaM {               // the same shared-memory slot as ChunkMeta
  float coef[kMaxCodeM + 1][kChunkSnpsM];    // (1 / N_i) / h_df, 0 for empty groups
  int32_t snp[kChunkSnpsM];                  // output SNP index, -1 = padding / left out
  uint16_t n[kMaxCodeM + 1][kChunkSnpsM];    // group sizes over non-missing samples
  uint8_t df[kChunkSnpsM];                   // non-empty groups - 1
  uint8_t pad_[1536 - 640 - 128 - 320 - 32];
};
static_assert(sizeof(ChunkMetaM) == sizeof(ChunkMeta), "ChunkMetaM must fill a ChunkMeta slot");

// Side record of a hit, written next to the public krux_hit record and used by the
// FP64 finalisation: the pair's group sizes and the group (cohort / bucket) index.
struct alignas(8) HitAux {
  uint16_t n0, n1, n2, group;
};

// Second side record of a hit on a marker with more than three groups: the
// sizes of groups 3 and 4 and the centred sums D_2, D_3 (D_4 follows).
struct alignas(16) HitAux2 {
  uint16_t n3, n4, pad0_, pad1_;
  int32_t d2, d3;
};

// Hit records move as one 16-byte and one 8-byte access (hit lists are 16-byte
// aligned; the host rejects other pointers).  Stores are streaming (evict-first):
// the records are not read again by the writing SM, and the scan kernel's small
// L1 (most of the unified memory is shared memory) should keep its own lines.
__device__ __forceinline__ void st_hit(krux_hit *dst, const krux_hit &r) {
  __stcs(reinterpret_cast<uint4 *>(dst), make_uint4(r.trait, r.snp, (uint32_t)r.d0, (uint32_t)r.d1));
}
__device__ __forceinline__ void st_aux(HitAux *dst, const HitAux &a) {
  __stcs(reinterpret_cast<uint2 *>(dst),
         make_uint2((uint32_t)a.n0 | ((uint32_t)a.n1 << 16), (uint32_t)a.n2 | ((uint32_t)a.group << 16)));
}
__device__ __forceinline__ krux_hit ld_hit(const krux_hit *src) {
  const uint4 v = *reinterpret_cast<const uint4 *>(src);
  krux_hit r;
  r.trait = v.x;
  r.snp = v.y;
  r.d0 = (int32_t)v.z;
  r.d1 = (int32_t)v.w;
  return r;
}
__device__ __forceinline__ HitAux ld_aux(const HitAux *src) {
  const uint2 v = *reinterpret_cast<const uint2 *>(src);
  HitAux a;
  a.n0 = (uint16_t)(v.x & 0xffffu);
  a.n1 = (uint16_t)(v.x >> 16);
  a.n2 = (uint16_t)(v.y & 0xffffu);
  a.group = (uint16_t)(v.y >> 16);
  return a;
}

// ---- rank set: everything the scan needs about one expression matrix ------
struct RankDev {
  __half *A;            // [rows_pad][Np] centred 2*rank (0 at NaN and padding)
  uint16_t *lo;         // [T][N] #present values strictly below (for bucket re-ranks)
  uint16_t *eq;         // [T][N] #present values equal (itself included), 0 at NaN
  int64_t *tie;         // [T] sum over present samples of eq^2 - 1 = sum (t^3 - t)
  int32_t *K;           // [T] present samples
  float *tau;           // [rows_pad] K(K+1)C/3 (fast-test bound), +inf when degenerate or padding
  double *cfac;         // [rows_pad] 3 / (K(K+1)C), 0 when degenerate or padding
  uint16_t *nan_cnt;    // [rows_pad] NaN samples of the trait (0 for padding)
  uint16_t *nan_idx;    // [T][N] their sample indices (first nan_cnt entries)
  uint32_t *tile_nan;   // [rows_pad/128] the tile's traits with NaN (low 16 bits) and
                        // with more than kNanCMax NaN samples (high 16 bits)
};

// One missing-pattern bucket of a scan call: the base rank set's ranks re-derived
// without the samples of the pattern (outputs per bucket; the NaN lists, counts
// and tile flags are the base set's own).
struct RerankJob {
  RankDev base;             // lo, eq, K and nan_cnt are read
  __half *A;                // [rows_pad][Np] (padding rows written as 0)
  int64_t *tie;             // [T]
  int32_t *K;               // [T]
  float *tau;               // [rows_pad]
  double *cfac;             // [rows_pad]
  int32_t T, N, Np, rows_pad;
  int32_t drop_off, n_drop; // the pattern's samples: drops[drop_off .. + n_drop)
};

// One SNP set of a batched packing launch (one scan group): slots
// [slot0, slot0 + 64 * nchunks) and, when the group needs genotype codes, chunk
// halves [half0, half0 + 2 * nchunks) of the flattened launch.
struct PackJob {
  const int8_t *geno;
  int64_t ldg;
  const int64_t *snp_list;  // device rows, or null for [snp_begin, snp_begin + n_snps)
  int64_t snp_begin, n_snps;
  int64_t slot0, half0;
  __half *B;
  ChunkMeta *meta;
  uint64_t *codes;          // null: no codes (and no halves)
  int32_t N, Np, allow_missing;
  int32_t coef_nan;         // 1: codes holds the plain form's coefficient blocks (kCoefNanBytes
                            // per chunk) instead of 2-bit codes
};

// ---- one group of a scan launch (a cohort, a missing-pattern bucket, or the
// unpermuted + permuted rank matrices of a permutation batch) ----------------
struct alignas(64) GroupDesc {
  CUtensorMap tmA;          // 2D fp16 [rowsA][Np], box {atom K, 128}, swizzled
  CUtensorMap tmB;          // 2D fp16 [nchunks*128][Np], box {atom K, 128}, swizzled
  const ChunkMeta *meta;    // [nchunks]
  const uint64_t *codes;    // [nchunks][Np][2] 2-bit genotype codes (3 = missing), or null
  const float *tau;         // [T]
  const double *cfac;       // [T]
  const uint16_t *nan_cnt;  // [T] or null when the rank set has no NaN
  const uint16_t *nan_idx;  // [T][N]
  const uint32_t *tile_nan; // [n_ttiles]
  krux_hit *hits;           // hit records (capacity entries)
  HitAux *aux;              // side records
  HitAux2 *aux2;            // second side records (markers with more than three groups)
  unsigned long long *counter;  // hits found (keeps counting past capacity)
  double *dense_H, *dense_p;    // optional [T][dense_ld]
  double *minp_key;         // permutation mode: [n_agroups-1][rows_per_agroup] best -ln p (as double bits)
  unsigned long long *minp_bound;  // plain-form permutations: [n_agroups-1][rows_per_agroup][2]
                            // (float bits of the largest decided df-1 |value| / df-2 value << 32)
                            // | identity of the pair that has it
  unsigned long long *minp_seed;  // their seed pass: [n_agroups-1][rows_per_agroup][2]
                            // (float bits of the largest value << 32) | (its 16-SNP block + 1)
  int64_t capacity;
  int64_t dense_ld;
  int64_t dense_snp0;       // SNP index of dense column 0
  int32_t T, N, Np, n_ttiles, rows_per_agroup, n_agroups, nchunks, n_atoms;
  int32_t group_id;
  int32_t nc;               // SNP chunks of one B tile (resident together)
  int32_t b_stride;         // shared-memory bytes of one resident B chunk
  int32_t nkb;              // rank-tile K blocks per step (1 = the whole K at once)
  int32_t pair;             // 1: chunks 2j, 2j+1 interleaved per K atom, one N = 256 MMA per pair
  int32_t codes_k;          // 16-byte rows of one chunk's codes block (Np, or kCoefNanRows
                            // for the plain form's NaN coefficient sets)
  int32_t a_row0, b_row0;   // first row of this group's A / B in tmA / tmB (maps may be shared)
  int64_t nan_ag_stride;    // elements between the NaN index lists of consecutive agroups
                            // (permuted groups: NaN samples sit at permuted positions)
  const int8_t *geno;       // plain form with NaN: the genotypes, for exact group sizes
  int64_t ldg;
};

// The plain form's hot-test coefficients for traits with NaN samples, one block
// per chunk (in place of the 2-bit codes): set s serves traits with up to
// kNanSetC[s] NaN samples, the same alpha (u + beta v)^2 + gamma v^2 form as
// ChunkMeta's first three arrays, built from group sizes max(N_i - C, 1) and the
// threshold of the smallest df the pair can keep, so that it bounds
// sum_i D_i^2 / N_i' / h_df' from above whatever genotypes the NaN samples carry
// (section "Handling missing values": N_i' counts the samples present for both).
// Traits with more NaN samples than the last set allows always reach the exact test.
constexpr int kNanSets = 5;
__host__ __device__ constexpr int nan_set_c(int s) { return s < 4 ? s + 1 : 6; }
__host__ __device__ constexpr int nan_set_of(int c) {  // -1: beyond the last set
  return c <= 4 ? c - 1 : (c <= 6 ? 4 : -1);
}
constexpr int kNanCMax = 6;
struct CoefSet {
  float alpha[kChunkSnps], beta[kChunkSnps], gamma[kChunkSnps];
};
// Set s starts at byte 16 (s + 1) + 768 s of a chunk's block: for one SNP the sets
// and the chunk metadata's coefficients then sit in different 16-byte bank groups
// of shared memory, and a warp whose lanes use different sets reads them in one pass.
constexpr int kCoefSetStride = (int)sizeof(CoefSet) + 16;
constexpr int kCoefNanBytes = 16 + kNanSets * kCoefSetStride;
constexpr int kCoefNanRows = kCoefNanBytes / 16;
static_assert(sizeof(CoefSet) == 768 && kCoefNanBytes % 16 == 0 && kCoefNanRows == 246,
              "coefficient block layout");
__host__ __device__ inline CoefSet *coef_set(void *block, int s) {
  return reinterpret_cast<CoefSet *>(static_cast<uint8_t *>(block) + 16 + s * kCoefSetStride);
}
__host__ __device__ inline const CoefSet *coef_set(const void *block, int s) {
  return reinterpret_cast<const CoefSet *>(static_cast<const uint8_t *>(block) + 16 +
                                           s * kCoefSetStride);
}

// Work item: B tile `btile` (chunks btile*nc .. +nc) of group `group`, against the
// (agroup, trait-tile) steps [step_begin, step_end) of that group.
struct WorkItem {
  int32_t group, btile, step_begin, step_end;
};

struct ScanParams {
  const GroupDesc *groups;
  const WorkItem *items;
  int32_t n_items;
  int32_t nc;               // most chunks any group keeps resident (<= kTmemSlots)
  int32_t nA;               // A pipeline stages
  int32_t kpad;             // widest K of the groups (codes rows are kpad * 16 bytes)
  int32_t ka;               // samples per A stage (a K block; multiple of the layout's atom)
  int32_t a_tile_bytes;     // 128 * ka * 2
  int32_t b_region;         // shared-memory bytes for the resident B chunks
  int32_t layout;           // 0: 128-byte swizzle, 64-element atoms; 1: 32-byte swizzle, 16-element atoms
  float margin;             // relative band rechecked in FP64
  int32_t dense;            // 1: every pair's H, p written in FP64
  double pthresh;
  float h1, h2;             // chi-square thresholds at pthresh for df 1, 2 (fp32)
  unsigned int *status;     // [0] error bits, [1] where
  long long timeout_cycles;
  int32_t signed_coef;      // 1: df-1 SNPs carry negated alpha, gamma (permutation batches)
  int32_t seg_cap;          // records per staging segment (0: hits go straight to the list)
  krux_hit *seg_hits;       // [grid][kEpiWarps][seg_cap] staged hit records, one segment per
                            // epilogue warp
  HitAux *seg_aux;          // [grid][kEpiWarps][seg_cap]
  unsigned int *seg_cnt;    // [grid][kEpiWarps] records staged in each segment
  unsigned long long *fdr_hist;  // permutation batches: [1 + P][fdr_bins] counts of p < P_c by
                                 // -log10 p bin (row 0 = real data, filled by the finalisation)
  int32_t fdr_bins;
  float fdr_pad_;
  double fdr_l0, fdr_w;     // bin b = floor((-log10 p - fdr_l0) / fdr_w), clamped to [0, bins)
  // cis mode (cis_window >= 0): a pair is reported only if |snp_pos - trait_pos| <= window
  const int64_t *cis_snp_pos;    // [S] global coordinate of every SNP row
  const int64_t *cis_trait_pos;  // [T] global coordinate of every trait (its gene)
  int64_t cis_window = -1;       // -1: off
  // markers with up to five groups (chunks of kChunkSnpsM SNPs, ChunkMetaM):
  int32_t multi = 0;
  HitAux2 *seg_aux2 = nullptr;   // [grid][kEpiWarps][seg_cap]
  // parametric comparison: every pair at or above the lower band edge is kept as
  // a provisional hit (decided later in FP64 from the FP32 values)
  int32_t provisional = 0;
  // permutation mode: some groups carry a min-p key (GroupDesc::minp_key)
  int32_t perm = 0;
  // seed pass of a permutation batch: the permuted groups write, per (permutation,
  // trait), a lower bound of the best -ln p over the scanned SNPs (no pair is decided)
  int32_t seed_bound = 0;
  // some group's rank set has NaN (its traits get the exact-size hot test)
  int32_t has_nan = 0;
  // plain-form permutation batches: each event warp's list of pairs for the
  // deferred FP64 pass ([grid][2][mc_cap]) and its count ([grid][2])
  MinpPair *mc_list = nullptr;
  unsigned int *mc_cnt = nullptr;
  int32_t mc_cap = 0;
  // the plain scan form applies: 32-byte swizzle, every group's chunks paired, no
  // dense output, no cis window, no provisional hits (permutation batches take its
  // two-sided variant; NaN in the expression its variant with coefficient sets,
  // fast_nan = 1, when at most one trait in 128 has more than kNanCMax NaN samples)
  int32_t fast = 0;
  int32_t fast_nan = 0;
};

enum : unsigned int {
  kDevTimeout = 1u,
  kDevBadCode = 2u,
  kDevBadPerm = 4u,     // a permutation entry outside 0..N-1 (its row is gathered as zeros)
  kDevMissing = 8u,     // a -1 code in a group packed as complete (graph replays)
  kDevHashCollision = 16u,  // two missing-sample patterns with one 64-bit hash
};

// ---- launch wrappers (defined in the .cu files) -----------------------------
cudaError_t launch_rank(const float *expr, int T, int N, int64_t ld, int Np, int rows_pad,
                        const RankDev &r, cudaStream_t s);
// NaN sample lists of the permuted rank matrices: out[q][t][j] = inv[q][nan_idx[t][j]]
// for j < nan_cnt[t] (sample k of permutation q takes the value of sample perm[q][k]).
cudaError_t launch_permute_nan_idx(const uint16_t *nan_cnt, const uint16_t *nan_idx, int T, int N,
                                   const int32_t *inv, int P, uint16_t *out, cudaStream_t s);
// inv[q][perms[q][k]] = k for every in-range entry.
cudaError_t launch_invert_perms(const int32_t *perms, int P, int N, int32_t *inv, cudaStream_t s);
// status (may be null) gets kDevBadPerm for an entry outside 0..N-1.
cudaError_t launch_permute_rows(const __half *A, __half *out, int rows_pad, int Np, int N,
                                const int32_t *perms, int P, unsigned int *status, cudaStream_t s);
cudaError_t launch_scan(const ScanParams &p, int grid, size_t smem, cudaStream_t s);
size_t scan_smem_bytes(int nc, int nA, int kpad);
size_t scan_smem_bytes2(int nc, int nA, size_t a_tile_bytes, size_t b_region, int codes_k);
cudaError_t launch_seg_compact(const krux_hit *seg_hits, const HitAux *seg_aux,
                               const HitAux2 *seg_aux2, const unsigned int *seg_cnt, int n_seg,
                               int seg_cap, const unsigned long long *direct, krux_hit *out,
                               HitAux *out_aux, HitAux2 *out_aux2, int64_t capacity,
                               unsigned long long *total, cudaStream_t s);
cudaError_t launch_minp_from_key(const double *key, double *minp, int P, int T, int ld,
                                 cudaStream_t s);
// Device-side grouping of the flagged SNPs by missing-sample pattern: scratch of
// one call (cap table slots, a power of two above twice the SNP count; per-SNP and
// per-bucket arrays of n_snps entries).
struct PatternScratch {
  unsigned long long *tab_hash;
  int *tab_rep, *tab_id, *slot_of, *bucket_of;
  unsigned int *n_buckets, *count, *fill;
  unsigned long long *first;  // smallest SNP row of each bucket
  uint64_t *bucket_mask;      // [bucket][kMaxN / 64]
  int64_t *offset;            // [bucket] list offsets (set by the host)
  int64_t *woff;              // [n_snps / 32 + 1] complete-row offsets
  int64_t cap;
};
cudaError_t launch_pattern_group(const unsigned int *n_missing, const uint64_t *mask,
                                 const int64_t *miss_idx, int64_t n_snps, PatternScratch &w,
                                 unsigned int *status, cudaStream_t s);
cudaError_t launch_pattern_lists(const unsigned int *n_missing, const int64_t *miss_idx,
                                 const uint32_t *flags, bool flags_ready, int64_t snp_begin,
                                 int64_t n_snps, PatternScratch &w, int64_t *bucket_list,
                                 int64_t *complete_list, cudaStream_t s);
// After a plain-form permutation launch: the FP64 -ln p of every pair the event
// warps passed on, folded into the keys and, in the FDR band, into the histogram.
cudaError_t launch_minp_cands(const MinpPair *list, const unsigned int *cnt, int n_lists, int cap,
                              const double *cfac, int rows_pad, double pthresh, double *key,
                              unsigned long long *fdr_hist, int fdr_bins, double fdr_l0,
                              double fdr_w, cudaStream_t s);
// After a plain-form seed pass: decides, per (permutation, trait, class), the pair
// with the seed's largest value exactly (see seed_decide_kernel).
cudaError_t launch_seed_decide(const unsigned long long *rec, const __half *stack, int rows_pad,
                               int Np, int N, int T, int P, const int8_t *geno, int64_t ldg,
                               int64_t snp_begin, int64_t n_snps, const ChunkMeta *meta,
                               const double *cfac, double *key, unsigned long long *bound,
                               cudaStream_t s);
cudaError_t launch_pad_traits(int T, int rows_pad, float *tau, double *cfac, uint16_t *nan_cnt,
                              cudaStream_t s);
// Uploads the 1/n table the finalisation uses (once per device; not during a
// graph capture).
cudaError_t finalize_prepare();
// Finalisation of min(*count, capacity) hits, the count read on the device;
// aux2 is non-null for markers with more than three groups.  pthresh: the hits'
// threshold P_c (a reported p at or above it is taken again in full FP64).
cudaError_t launch_finalize_dev(const krux_hit *hits, const HitAux *aux, const HitAux2 *aux2,
                                const unsigned long long *count, int64_t capacity,
                                const double *const *cfac_by_group, double *H, double *p,
                                int sm_count, cudaStream_t s, unsigned long long *fdr_hist,
                                int fdr_bins, double fdr_l0, double fdr_w, double pthresh);
cudaError_t scan_set_smem(size_t smem);
int scan_form_of(const ScanParams &p);
cudaError_t launch_scan_only(const ScanParams &p, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_finalize(const krux_hit *hits, const HitAux *aux, int64_t n,
                            const double *const *cfac_by_group, double *H, double *p,
                            cudaStream_t s, unsigned long long *fdr_hist, int fdr_bins,
                            double fdr_l0, double fdr_w, double pthresh);

}  // namespace krux
