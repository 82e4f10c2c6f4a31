// pack.cu -- genotype packing (section "Calculation of the Kruskal-Wallis test
// statistic by matrix multiplication": the index matrices I_i(m,k) = [G(m,k) = i]
// and the group sizes N_i(m) = sum_k I_i(m,k)).
//
// Only I_0 and I_1 are materialised: with centred ranks the three rank sums
// satisfy D_0 + D_1 + D_2 = 0, so D_2 follows from the other two.  The packed
// operand is FP16 0/1 in chunks of 64 SNPs: chunk c holds rows [0,64) = I_0 and
// rows [64,128) = I_1 of SNPs 64c .. 64c+63, each row Np samples long.
#include "common.cuh"

namespace krux {

namespace {
constexpr int kPackWarps = 8;

// Missing-genotype pre-pass: flags SNPs with a -1 code, appends (index, sample
// bitmask) of each such SNP, and reports codes outside {-1, 0..max_code}.
__global__ void __launch_bounds__(kPackWarps * 32)
missing_scan_kernel(const int8_t *__restrict__ geno, int64_t ldg, int N, int64_t snp_begin,
                    int64_t n_snps, int max_code, unsigned int *n_missing, int64_t *miss_idx,
                    uint64_t *miss_mask, unsigned int *status) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t j = (int64_t)blockIdx.x * kPackWarps + warp;
  if (j >= n_snps) return;
  const int8_t *g = geno + (snp_begin + j) * ldg;
  uint32_t words[kMaxN / 32];
  bool any = false, bad = false;
#pragma unroll
  for (int w = 0; w < kMaxN / 32; ++w) {
    words[w] = 0u;
    if (w * 32 < N) {  // warp-uniform
      const int k = w * 32 + lane;
      const int code = k < N ? (int)g[k] : 0;
      bad |= (code < -1 || code > max_code);
      words[w] = __ballot_sync(0xffffffffu, code == -1);
      any |= words[w] != 0u;
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, kDevBadCode);
  if (!any) return;
  unsigned int slot = 0;
  if (lane == 0) slot = atomicAdd(n_missing, 1u);
  slot = __shfl_sync(0xffffffffu, slot, 0);
  if (lane == 0) miss_idx[slot] = snp_begin + j;
  if (lane < kMaxN / 64) {
    const uint64_t m = (uint64_t)words[2 * lane] | ((uint64_t)words[2 * lane + 1] << 32);
    miss_mask[(int64_t)slot * (kMaxN / 64) + lane] = m;
  }
}

// The same pre-pass for rows stored back to back (ldg == N), which is the usual
// layout: the block is read as a flat byte array with 16-byte loads, every byte
// checked four at a time; a -1 sets the bit of its SNP in `flags` (rare), a code
// outside {-1, 0..max_code} sets kDevBadCode.  base = row 0 of the range, nbytes
// = rows * N.
__device__ __forceinline__ void missing_word(uint32_t x, int64_t o, int N, uint32_t mc4,
                                             uint32_t *flags, bool &bad) {
  uint32_t ff = __vcmpeq4(x, 0xffffffffu);
  bad |= (__vcmpgtu4(x, mc4) & ~ff) != 0u;
  while (ff != 0u) {
    const int byte = (__ffs(ff) - 1) >> 3;
    const int64_t snp = (o + byte) / N;
    atomicOr(&flags[snp >> 5], 1u << (snp & 31));
    ff &= ~(0xffu << (8 * byte));
  }
}

__global__ void __launch_bounds__(256)
missing_flag_kernel(const int8_t *__restrict__ base, int64_t nbytes, int N, int max_code,
                    uint32_t *flags, unsigned int *status) {
  const uint32_t mc4 = (uint32_t)max_code * 0x01010101u;
  const int64_t head = std::min<int64_t>((16 - (int64_t)((uintptr_t)base & 15)) & 15, nbytes);
  const int64_t words = (nbytes - head) / 16;
  const int64_t tail0 = head + 16 * words;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  bool bad = false;
  for (int64_t i = tid; i < words; i += nthreads) {
    const uint4 v = *reinterpret_cast<const uint4 *>(base + head + 16 * i);
    const int64_t o = head + 16 * i;
    missing_word(v.x, o, N, mc4, flags, bad);
    missing_word(v.y, o + 4, N, mc4, flags, bad);
    missing_word(v.z, o + 8, N, mc4, flags, bad);
    missing_word(v.w, o + 12, N, mc4, flags, bad);
  }
  // the unaligned head and the tail, one byte per thread
  const int64_t extra = head + (nbytes - tail0);
  if (tid < extra) {
    const int64_t o = tid < head ? tid : tail0 + (tid - head);
    const int code = base[o];
    if (code == -1) {
      const int64_t snp = o / N;
      atomicOr(&flags[snp >> 5], 1u << (snp & 31));
    }
    bad |= code < -1 || code > max_code;
  }
  if (bad) atomicOr(status, kDevBadCode);
}

// The flagged SNPs (bit j of flags: SNP snp_begin + j) appended as (index, sample
// bitmask), one warp per flag word.
__global__ void __launch_bounds__(256)
missing_collect_kernel(const int8_t *__restrict__ geno, int64_t ldg, int N, int64_t snp_begin,
                       int64_t n_snps, const uint32_t *__restrict__ flags, unsigned int *n_missing,
                       int64_t *miss_idx, uint64_t *miss_mask) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t w = (int64_t)blockIdx.x * 8 + warp;
  if (w * 32 >= n_snps) return;
  uint32_t bits = flags[w];
  while (bits != 0u) {
    const int bit = __ffs(bits) - 1;
    bits &= bits - 1u;
    const int64_t j = w * 32 + bit;
    const int8_t *g = geno + (snp_begin + j) * ldg;
    uint32_t words[kMaxN / 32];
#pragma unroll
    for (int q = 0; q < kMaxN / 32; ++q) {
      words[q] = 0u;
      if (q * 32 < N) {  // warp-uniform
        const int k = q * 32 + lane;
        words[q] = __ballot_sync(0xffffffffu, k < N && g[k] == -1);
      }
    }
    unsigned int slot = 0;
    if (lane == 0) slot = atomicAdd(n_missing, 1u);
    slot = __shfl_sync(0xffffffffu, slot, 0);
    if (lane == 0) miss_idx[slot] = snp_begin + j;
    if (lane < kMaxN / 64) {
      const uint64_t m = (uint64_t)words[2 * lane] | ((uint64_t)words[2 * lane + 1] << 32);
      miss_mask[(int64_t)slot * (kMaxN / 64) + lane] = m;
    }
  }
}

// ---- device-side grouping of the flagged SNPs by missing-sample pattern ----------
// (section "Handling missing values": one matrix per pattern).  An open-addressing
// table over 64-bit hashes of the sample masks (0 = empty slot) finds each pattern's
// bucket; every member's mask is then compared with its bucket representative's
// (a hash collision is reported, and the host groups on its own instead).
__device__ __forceinline__ uint64_t pattern_hash(const uint64_t *m) {
  uint64_t h = 0x9e3779b97f4a7c15ull;
#pragma unroll
  for (int w = 0; w < kMaxN / 64; ++w) h = (h ^ m[w]) * 0x100000001b3ull;
  return (h ^ (h >> 29)) | 1ull;
}

__global__ void pattern_insert_kernel(const unsigned int *__restrict__ n_missing,
                                      const uint64_t *__restrict__ mask,
                                      unsigned long long *tab_hash, int *tab_rep, int64_t cap,
                                      int *slot_of) {
  const int64_t m = *n_missing;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long h = pattern_hash(mask + i * (kMaxN / 64));
    int64_t t = (int64_t)(h & (unsigned long long)(cap - 1));
    for (int64_t probe = 0; probe < cap; ++probe) {  // the table has room for every mask
      const unsigned long long prev = atomicCAS(tab_hash + t, 0ull, h);
      if (prev == 0ull || prev == h) {
        atomicMin(tab_rep + t, (int)i);
        slot_of[i] = (int)t;
        break;
      }
      t = (t + 1) & (cap - 1);
    }
  }
}

// Numbers the occupied slots (bucket ids) and copies each bucket's representative
// mask out.
__global__ void pattern_number_kernel(const unsigned long long *__restrict__ tab_hash,
                                      const int *__restrict__ tab_rep, int64_t cap, int *tab_id,
                                      unsigned int *n_buckets, const uint64_t *__restrict__ mask,
                                      uint64_t *bucket_mask) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cap;
       t += (int64_t)gridDim.x * blockDim.x) {
    if (tab_hash[t] == 0ull) continue;
    const int id = (int)atomicAdd(n_buckets, 1u);
    tab_id[t] = id;
    const int rep = tab_rep[t];
#pragma unroll
    for (int w = 0; w < kMaxN / 64; ++w)
      bucket_mask[(int64_t)id * (kMaxN / 64) + w] = mask[(int64_t)rep * (kMaxN / 64) + w];
  }
}

// Bucket of every flagged SNP, bucket sizes and first SNPs, and the check of every
// mask against its bucket's.
__global__ void pattern_count_kernel(const unsigned int *__restrict__ n_missing,
                                     const int *__restrict__ slot_of, const int *__restrict__ tab_id,
                                     const uint64_t *__restrict__ mask,
                                     const uint64_t *__restrict__ bucket_mask,
                                     const int64_t *__restrict__ miss_idx, int *bucket_of,
                                     unsigned int *count, unsigned long long *first,
                                     unsigned int *status) {
  const int64_t m = *n_missing;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int b = tab_id[slot_of[i]];
    bucket_of[i] = b;
    atomicAdd(count + b, 1u);
    atomicMin(first + b, (unsigned long long)miss_idx[i]);
    bool same = true;
#pragma unroll
    for (int w = 0; w < kMaxN / 64; ++w)
      same = same && mask[i * (kMaxN / 64) + w] == bucket_mask[(int64_t)b * (kMaxN / 64) + w];
    if (!same) atomicOr(status, kDevHashCollision);
  }
}

// Writes every flagged SNP into its bucket's list (offset[b] .. + count[b]).
__global__ void pattern_scatter_kernel(const unsigned int *__restrict__ n_missing,
                                       const int *__restrict__ bucket_of,
                                       const int64_t *__restrict__ offset,
                                       const int64_t *__restrict__ miss_idx, unsigned int *fill,
                                       int64_t *list) {
  const int64_t m = *n_missing;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int b = bucket_of[i];
    list[offset[b] + atomicAdd(fill + b, 1u)] = miss_idx[i];
  }
}

// The rows without a missing code, in order: one block scans the per-word counts of
// the flag bits, then every word writes its complete rows.
__global__ void __launch_bounds__(1024)
complete_offsets_kernel(const uint32_t *__restrict__ flags, int64_t n_snps, int64_t *woff) {
  __shared__ int64_t part[1024];
  const int64_t nw = (n_snps + 31) / 32;
  const int64_t per = (nw + 1023) / 1024;
  const int64_t w0 = threadIdx.x * per, w1 = w0 + per < nw ? w0 + per : nw;
  int64_t sum = 0;
  for (int64_t w = w0; w < w1; ++w) {
    const int64_t left = n_snps - 32 * w;
    const int valid = left < 32 ? (int)left : 32;
    const uint32_t vm = valid >= 32 ? 0xffffffffu : (1u << valid) - 1u;
    sum += __popc(~flags[w] & vm);
  }
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int d = 1; d < 1024; d <<= 1) {  // inclusive scan of the partial sums
    const int64_t v = threadIdx.x >= (unsigned)d ? part[threadIdx.x - d] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int64_t run = threadIdx.x ? part[threadIdx.x - 1] : 0;
  for (int64_t w = w0; w < w1; ++w) {
    woff[w] = run;
    const int64_t left = n_snps - 32 * w;
    const int valid = left < 32 ? (int)left : 32;
    const uint32_t vm = valid >= 32 ? 0xffffffffu : (1u << valid) - 1u;
    run += __popc(~flags[w] & vm);
  }
  if (threadIdx.x == 1023) woff[nw] = part[1023];
}

__global__ void complete_scatter_kernel(const uint32_t *__restrict__ flags,
                                        const int64_t *__restrict__ woff, int64_t snp_begin,
                                        int64_t n_snps, int64_t *list) {
  const int64_t nw = (n_snps + 31) / 32;
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nw;
       w += (int64_t)gridDim.x * blockDim.x) {
    const int64_t left = n_snps - 32 * w;
    const int valid = left < 32 ? (int)left : 32;
    uint32_t bits = ~flags[w] & (valid >= 32 ? 0xffffffffu : (1u << valid) - 1u);
    int64_t o = woff[w];
    while (bits) {
      const int j = __ffs((int)bits) - 1;
      bits &= bits - 1u;
      list[o++] = snp_begin + 32 * w + j;
    }
  }
}

// Flag bits of the flagged SNPs (the pre-pass that produces no flag array).
__global__ void flags_from_idx_kernel(const unsigned int *__restrict__ n_missing,
                                      const int64_t *__restrict__ miss_idx, int64_t snp_begin,
                                      uint32_t *flags) {
  const int64_t m = *n_missing;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = miss_idx[i] - snp_begin;
    atomicOr(flags + (j >> 5), 1u << (j & 31));
  }
}

// Metadata of SNP slot jj of a chunk: group sizes, df and the coefficients of the
// hot test (zero for an excluded SNP: one with a missing code outside its bucket).
__device__ __forceinline__ void write_meta(ChunkMeta &m, int jj, int n0, int n1, int n2,
                                           bool excluded, int64_t snp_out, float rh1, float rh2,
                                           int signed_df1, int linear, float rl) {
  const int groups = (n0 > 0) + (n1 > 0) + (n2 > 0);
  const int df = groups > 0 ? groups - 1 : 0;
  float al = 0.f, be = 0.f, ga = 0.f;
  if (linear) {
    // dosage regression (parametric comparison): rl (2 S_0 + S_1)^2 / S_gg,
    // S_gg = sum over samples of (g - mean g)^2
    const int K = n0 + n1 + n2;
    const float gs = (float)n1 + 2.f * (float)n2;
    const float sgg = K > 0 ? (float)n1 + 4.f * (float)n2 - gs * gs / (float)K : 0.f;
    if (df > 0 && !excluded && sgg > 0.5f / (float)(K > 0 ? K : 1)) {
      al = 4.f * rl / sgg;
      be = 0.5f;
    }
  } else if (df > 0 && !excluded) {
    // sum_i D_i^2 / N_i with D_2 = -(u + v):  (r0 + r2) u^2 + 2 r2 u v + (r1 + r2) v^2
    //   = alpha (u + beta v)^2 + gamma v^2,  alpha = r0 + r2, beta = r2 / alpha,
    //   gamma = r1 + r2 r0 / alpha   (empty groups have r_i = 0).  FP32 is enough:
    // these only feed the thresholded test, whose band is rechecked in FP64.
    const float q0 = n0 ? 1.f / (float)n0 : 0.f, q1 = n1 ? 1.f / (float)n1 : 0.f,
                q2 = n2 ? 1.f / (float)n2 : 0.f;
    const float a = q0 + q2;
    const float rh = (df == 1 ? rh1 : rh2) * ((signed_df1 && df == 1) ? -1.f : 1.f);
    al = a * rh;
    be = q2 / a;
    ga = (q1 + q2 * q0 / a) * rh;
  }
  m.alpha[jj] = al;
  m.beta[jj] = be;
  m.gamma[jj] = ga;
  m.snp[jj] = excluded ? -1 : (int32_t)snp_out;
  m.n[0][jj] = (uint16_t)n0;
  m.n[1][jj] = (uint16_t)n1;
  m.n[2][jj] = (uint16_t)n2;
  m.df[jj] = (uint8_t)df;
}

// The plain form's coefficient sets of SNP slot jj for traits with NaN samples:
// set s takes write_meta's alpha, beta, gamma from group sizes max(N_i - C, 1),
// C = nan_set_c(s) (an empty group stays empty), with the threshold of the
// smallest df the pair can keep (1/h_1 when some group may vanish).  For a trait
// with c <= C NaN samples they bound the pair's exact sum_i D_i^2 / N_i' / h_df'
// from above, whichever groups the NaN samples fall in.
__device__ __forceinline__ void write_coef_nan(void *block, int jj, int n0, int n1, int n2,
                                               bool excluded, float rh1, float rh2) {
  const int groups = (n0 > 0) + (n1 > 0) + (n2 > 0);
#pragma unroll
  for (int si = 0; si < kNanSets; ++si) {
    const int c = nan_set_c(si);
    float al = 0.f, be = 0.f, ga = 0.f;
    if (groups > 1 && !excluded) {
      const int sure = (n0 > c) + (n1 > c) + (n2 > c);  // groups no c NaN samples can empty
      const float rh = sure >= 3 ? rh2 : rh1;
      const float q0 = n0 ? 1.f / (float)max(n0 - c, 1) : 0.f, q1 = n1 ? 1.f / (float)max(n1 - c, 1) : 0.f,
                  q2 = n2 ? 1.f / (float)max(n2 - c, 1) : 0.f;
      const float a = q0 + q2;
      if (a > 0.f) {
        al = a * rh;
        be = q2 / a;
        ga = (q1 + q2 * q0 / a) * rh;
      } else {
        ga = q1 * rh;  // groups 0 and 2 empty (cannot happen with two groups or more)
      }
    }
    CoefSet *cs = coef_set(block, si);
    cs->alpha[jj] = al;
    cs->beta[jj] = be;
    cs->gamma[jj] = ga;
  }
}

// Packs SNP slot j (one warp; j may be the padding of the last chunk).  SNP j is
// snp_list[j] if a list is given, else snp_begin + j.  SNPs that carry a missing
// code are packed with zero coefficients here (they are scanned in their
// missing-pattern bucket, where the rank set excludes those samples and the -1
// entries simply pack as 0 in both indicators).
__device__ __forceinline__ void pack_slot(const int8_t *__restrict__ geno, int64_t ldg, int N,
                                          int Np, const int64_t *__restrict__ snp_list,
                                          int64_t snp_begin, int64_t n_snps, int64_t j,
                                          int64_t snp_out_base, float rh1, float rh2,
                                          int allow_missing, int signed_df1,
                                          __half *__restrict__ B, ChunkMeta *__restrict__ meta,
                                          unsigned int *status, int linear, float rl, int lane) {
  const int64_t c = j / kChunkSnps;
  const int jj = (int)(j % kChunkSnps);
  __half *r0 = B + (c * kChunkRows + jj) * Np;
  __half *r1 = B + (c * kChunkRows + kChunkSnps + jj) * Np;
  ChunkMeta &m = meta[c];
  const __half one = __int2half_rn(1), zero = __int2half_rn(0);
  if (j >= n_snps) {
    for (int k = lane; k < Np; k += 32) {
      r0[k] = zero;
      r1[k] = zero;
    }
    if (lane == 0) {
      m.alpha[jj] = 0.f;
      m.beta[jj] = 0.f;
      m.gamma[jj] = 0.f;
      m.snp[jj] = -1;
      m.n[0][jj] = m.n[1][jj] = m.n[2][jj] = 0;
      m.df[jj] = 0;
    }
    return;
  }
  const int64_t s = snp_list ? snp_list[j] : snp_begin + j;
  const int8_t *g = geno + s * ldg;
  int n0 = 0, n1 = 0, n2 = 0;
  bool miss = false, bad = false;
  for (int k = lane; k < Np; k += 32) {
    const int code = k < N ? (int)g[k] : -1;
    r0[k] = code == 0 ? one : zero;
    r1[k] = code == 1 ? one : zero;
    n0 += code == 0;
    n1 += code == 1;
    n2 += code == 2;
    if (k < N) {
      miss |= code == -1;
      bad |= (code < -1 || code > 2);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    n0 += __shfl_xor_sync(0xffffffffu, n0, o);
    n1 += __shfl_xor_sync(0xffffffffu, n1, o);
    n2 += __shfl_xor_sync(0xffffffffu, n2, o);
  }
  miss = __any_sync(0xffffffffu, miss);
  bad = __any_sync(0xffffffffu, bad);
  if (lane == 0) {
    if (bad) atomicOr(status, kDevBadCode);
    if (miss && !allow_missing) atomicOr(status, kDevMissing);
    write_meta(m, jj, n0, n1, n2, miss && !allow_missing, snp_out_base + s, rh1, rh2, signed_df1,
               linear, rl);
  }
}

// One warp per packed SNP slot of one SNP set.
__global__ void __launch_bounds__(kPackWarps * 32)
pack_kernel(const int8_t *__restrict__ geno, int64_t ldg, int N, int Np,
            const int64_t *__restrict__ snp_list, int64_t snp_begin, int64_t n_snps,
            int64_t n_slots, int64_t snp_out_base, float rh1, float rh2, int allow_missing,
            int signed_df1, __half *__restrict__ B, ChunkMeta *__restrict__ meta,
            unsigned int *status, int linear, float rl) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t j = (int64_t)blockIdx.x * kPackWarps + warp;
  if (j >= n_slots) return;
  pack_slot(geno, ldg, N, Np, snp_list, snp_begin, n_snps, j, snp_out_base, rh1, rh2,
            allow_missing, signed_df1, B, meta, status, linear, rl, lane);
}

// Last job whose first flattened unit is at or below x (x below the total).
__device__ __forceinline__ int find_job(const PackJob *__restrict__ jobs, int n_jobs, int64_t x,
                                        bool halves) {
  int lo = 0, hi = n_jobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((halves ? jobs[mid].half0 : jobs[mid].slot0) <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Staged packing of 32 consecutive genotype rows of at most kStageLd bytes each
// (no SNP list): the warp copies the rows' byte span into shared memory with
// 16-byte loads, writes both indicator blocks (32 rows of I_0, then 32 of I_1, each
// contiguous) with 16-byte stores, and lane i counts the groups of row i.
constexpr int kStageLd = 128;
constexpr int kStageBytes = 32 * kStageLd + 32;

// Four codes starting at byte offset o of the staged span (any alignment).
__device__ __forceinline__ uint32_t stage_word(const uint8_t *st, int o) {
  const uint32_t *w = reinterpret_cast<const uint32_t *>(st + (o & ~3));
  return __funnelshift_r(w[0], w[1], 8 * (o & 3));
}
// Bytes 0..3 of a 0x00 / 0xff byte mask as two FP16 pairs (1.0 where 0xff).
__device__ __forceinline__ uint2 mask_to_halves(uint32_t m) {
  return make_uint2(__byte_perm(m, 0u, 0x1100) & 0x3c003c00u, __byte_perm(m, 0u, 0x3322) & 0x3c003c00u);
}

__device__ __forceinline__ void pack_staged(const PackJob &J, int64_t j0, uint8_t *st, int lane,
                                            int &my_n0, int &my_n1, int &my_n2, bool &my_miss,
                                            bool &any_bad, int64_t &my_s) {
  const int N = J.N, Np = J.Np;
  const int64_t ldg = J.ldg;
  const int64_t left = J.n_snps - j0;
  const int rows = left < 32 ? (int)left : 32;
  const uint8_t *src = reinterpret_cast<const uint8_t *>(J.geno + (J.snp_begin + j0) * ldg);
  // the span [src, src + L) in shared memory at offset pad + b, so that 16-byte
  // aligned global chunks land on 16-byte aligned shared addresses
  const int64_t L = (int64_t)(rows - 1) * ldg + N;
  const int pad = (int)((uintptr_t)src & 15u);
  const int head = (16 - pad) & 15;
  const int64_t mid = L > head ? (L - head) / 16 : 0;
  const int64_t hl = (int64_t)head < L ? (int64_t)head : L;
  for (int64_t b = lane; b < hl; b += 32) st[pad + b] = src[b];
  for (int64_t c = lane; c < mid; c += 32)
    *reinterpret_cast<uint4 *>(st + pad + head + 16 * c) =
        *reinterpret_cast<const uint4 *>(src + head + 16 * c);
  for (int64_t b = head + 16 * mid + lane; b < L; b += 32) st[pad + b] = src[b];
  __syncwarp();
  // both indicator blocks: item t = row r, samples 8q .. 8q + 7
  const int c = (int)(j0 / kChunkSnps), jj0 = (int)(j0 % kChunkSnps);
  const int per_row = Np / 8;
  uint4 *d0 = reinterpret_cast<uint4 *>(J.B + ((int64_t)c * kChunkRows + jj0) * Np);
  uint4 *d1 = reinterpret_cast<uint4 *>(J.B + ((int64_t)c * kChunkRows + kChunkSnps + jj0) * Np);
  for (int t = lane; t < 32 * per_row; t += 32) {
    const int r = t / per_row, k8 = 8 * (t - r * per_row);
    uint32_t lo = 0x03030303u, hi = 0x03030303u;  // 3: neither group 0 nor 1
    if (r < rows) {
      const int o = pad + (int)(r * ldg) + k8;
      lo = stage_word(st, o);
      hi = stage_word(st, o + 4);
      // samples at or beyond N are padding
      const int vl = min(max(N - k8, 0), 4), vh = min(max(N - k8 - 4, 0), 4);
      const uint32_t ml = vl >= 4 ? 0xffffffffu : (1u << (8 * vl)) - 1u;
      const uint32_t mh = vh >= 4 ? 0xffffffffu : (1u << (8 * vh)) - 1u;
      lo = (lo & ml) | (0x03030303u & ~ml);
      hi = (hi & mh) | (0x03030303u & ~mh);
    }
    const uint2 a = mask_to_halves(__vcmpeq4(lo, 0u)), b = mask_to_halves(__vcmpeq4(hi, 0u));
    const uint2 e = mask_to_halves(__vcmpeq4(lo, 0x01010101u)),
                f = mask_to_halves(__vcmpeq4(hi, 0x01010101u));
    d0[t] = make_uint4(a.x, a.y, b.x, b.y);
    d1[t] = make_uint4(e.x, e.y, f.x, f.y);
  }
  // lane i: the group sizes, missing and invalid codes of row i
  if (lane < rows) {
    int n0 = 0, n1 = 0, n2 = 0, nm = 0;
    const int o0 = pad + (int)(lane * ldg);
    for (int k = 0; k < N; k += 4) {
      uint32_t w = stage_word(st, o0 + k);
      const int v = min(N - k, 4);
      const uint32_t m = v >= 4 ? 0xffffffffu : (1u << (8 * v)) - 1u;
      w = (w & m) | (0x04040404u & ~m);  // 4: outside every class below
      n0 += __popc(__vcmpeq4(w, 0u)) >> 3;
      n1 += __popc(__vcmpeq4(w, 0x01010101u)) >> 3;
      n2 += __popc(__vcmpeq4(w, 0x02020202u)) >> 3;
      nm += __popc(__vcmpeq4(w, 0xffffffffu)) >> 3;
    }
    my_n0 = n0;
    my_n1 = n1;
    my_n2 = n2;
    my_miss = nm > 0;
    any_bad = n0 + n1 + n2 + nm != N;
    my_s = J.snp_begin + j0 + lane;
  }
  __syncwarp();
}

// All SNP sets of a call in one launch (rank-sum form): one warp per 32 flattened
// slots (half a chunk; every job spans whole chunks).  Lane t writes samples
// 4t .. 4t + 3 (+ 128 per pass) of both indicator rows of each slot with 8-byte
// stores, the group sizes come from warp reductions, and lane i then writes the
// metadata of slot i, so no lane does the per-SNP scalar work alone.
__global__ void __launch_bounds__(kPackWarps * 32)
pack_batch_kernel(const PackJob *__restrict__ jobs, int n_jobs, int64_t total_slots, float rh1,
                  float rh2, int signed_df1, unsigned int *status) {
  __shared__ __align__(16) uint8_t stage[kPackWarps][kStageBytes];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t x0 = ((int64_t)blockIdx.x * kPackWarps + warp) * 32;
  if (x0 >= total_slots) return;
  const PackJob &J = jobs[find_job(jobs, n_jobs, x0, false)];
  const int64_t j0 = x0 - J.slot0;  // a multiple of 32
  const int N = J.N, Np = J.Np;
  if (!J.snp_list && J.ldg <= kStageLd && Np <= kStageLd && j0 < J.n_snps) {
    int n0 = 0, n1 = 0, n2 = 0;
    bool miss = false, bad = false;
    int64_t sn = -1;
    pack_staged(J, j0, stage[warp], lane, n0, n1, n2, miss, bad, sn);
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, kDevBadCode);
    const bool excl = miss && !J.allow_missing;
    if (__any_sync(0xffffffffu, excl) && lane == 0) atomicOr(status, kDevMissing);
    ChunkMeta &m = J.meta[j0 / kChunkSnps];
    const int jj = (int)(j0 % kChunkSnps) + lane;
    if (sn < 0) write_meta(m, jj, 0, 0, 0, true, 0, rh1, rh2, signed_df1, 0, 0.f);
    else write_meta(m, jj, n0, n1, n2, excl, sn, rh1, rh2, signed_df1, 0, 0.f);
    if (J.coef_nan)
      write_coef_nan(reinterpret_cast<uint8_t *>(J.codes) + (j0 / kChunkSnps) * kCoefNanBytes, jj, sn < 0 ? 0 : n0,
                     sn < 0 ? 0 : n1, sn < 0 ? 0 : n2, sn < 0 || excl, rh1, rh2);
    return;
  }
  const int64_t c = j0 / kChunkSnps;
  const int jj0 = (int)(j0 % kChunkSnps);
  const uint32_t one2 = 0x3c003c00u;  // two FP16 ones
  // the job's arrays through restrict pointers: the genotype reads of a slot may
  // then be issued before the previous slot's stores
  const int8_t *__restrict__ geno = J.geno;
  const int64_t *__restrict__ snp_list = J.snp_list;
  __half *__restrict__ Bj = J.B;
  const int64_t ldg = J.ldg, n_snps = J.n_snps, snp_begin = J.snp_begin;
  int my_n0 = 0, my_n1 = 0, my_n2 = 0;
  bool my_miss = false, any_bad = false;
  int64_t my_s = 0;
#pragma unroll 2
  for (int i = 0; i < 32; ++i) {
    const int64_t j = j0 + i;
    const bool valid = j < n_snps;
    const int64_t s = valid ? (snp_list ? snp_list[j] : snp_begin + j) : 0;
    const int8_t *g = geno + s * ldg;
    __half *r0 = Bj + (c * kChunkRows + jj0 + i) * Np;
    __half *r1 = Bj + (c * kChunkRows + kChunkSnps + jj0 + i) * Np;
    int n0 = 0, n1 = 0, n2 = 0;
    bool miss = false, bad = false;
    for (int k0 = 4 * lane; k0 < Np; k0 += 128) {
      uint32_t h0[2] = {0u, 0u}, h1[2] = {0u, 0u};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = k0 + q;
        const int code = (valid && k < N) ? (int)g[k] : -1;
        const uint32_t bit = (q & 1) ? 0xffff0000u : 0x0000ffffu;
        if (code == 0) h0[q >> 1] |= one2 & bit;
        if (code == 1) h1[q >> 1] |= one2 & bit;
        n0 += code == 0;
        n1 += code == 1;
        n2 += code == 2;
        if (valid && k < N) {
          miss |= code == -1;
          bad |= (code < -1 || code > 2);
        }
      }
      *reinterpret_cast<uint2 *>(r0 + k0) = make_uint2(h0[0], h0[1]);
      *reinterpret_cast<uint2 *>(r1 + k0) = make_uint2(h1[0], h1[1]);
    }
    n0 = (int)__reduce_add_sync(0xffffffffu, (unsigned)n0);
    n1 = (int)__reduce_add_sync(0xffffffffu, (unsigned)n1);
    n2 = (int)__reduce_add_sync(0xffffffffu, (unsigned)n2);
    miss = __any_sync(0xffffffffu, miss);
    any_bad |= bad;
    if (lane == i) {
      my_n0 = valid ? n0 : 0;
      my_n1 = valid ? n1 : 0;
      my_n2 = valid ? n2 : 0;
      my_miss = miss;
      my_s = valid ? s : -1;
    }
  }
  if (__any_sync(0xffffffffu, any_bad) && lane == 0) atomicOr(status, kDevBadCode);
  const bool excl = my_miss && !J.allow_missing;
  if (__any_sync(0xffffffffu, excl) && lane == 0) atomicOr(status, kDevMissing);
  ChunkMeta &m = J.meta[c];
  if (my_s < 0) {  // padding slot of the last chunk
    write_meta(m, jj0 + lane, 0, 0, 0, true, 0, rh1, rh2, signed_df1, 0, 0.f);
  } else {
    write_meta(m, jj0 + lane, my_n0, my_n1, my_n2, excl, my_s, rh1, rh2, signed_df1, 0, 0.f);
  }
  if (J.coef_nan)
    write_coef_nan(reinterpret_cast<uint8_t *>(J.codes) + c * kCoefNanBytes, jj0 + lane, my_s < 0 ? 0 : my_n0,
                   my_s < 0 ? 0 : my_n1, my_s < 0 ? 0 : my_n2, my_s < 0 || excl, rh1, rh2);
}

__device__ __forceinline__ uint64_t spread_bits(uint32_t v) {
  uint64_t x = v;
  x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
  x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
  x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
  x = (x | (x << 2)) & 0x3333333333333333ull;
  x = (x | (x << 1)) & 0x5555555555555555ull;
  return x;
}

// 2-bit genotype codes per chunk and sample: word [c][k][h] holds, at bits
// 2j..2j+1, the code of SNP 64c + 32h + j at sample k (0,1,2; 3 = missing or
// padding).  Used by the epilogue to drop a trait's NaN samples from N_i.  One
// warp per chunk half hw = 2c + h.
__device__ __forceinline__ void codes_half(const int8_t *__restrict__ geno, int64_t ldg, int N,
                                           int Np, const int64_t *__restrict__ snp_list,
                                           int64_t snp_begin, int64_t n_snps, int64_t hw,
                                           uint64_t *__restrict__ codes, int lane) {
  const int64_t j = hw * 32 + lane;
  const int8_t *g = nullptr;
  if (j < n_snps) g = geno + (snp_list ? snp_list[j] : snp_begin + j) * ldg;
  const int64_t c = hw >> 1;
  const int h = (int)(hw & 1);
  for (int k = 0; k < Np; ++k) {
    int code = 3;
    if (g && k < N) {
      const int v = g[k];
      code = (v >= 0 && v <= 2) ? v : 3;
    }
    const uint32_t b0 = __ballot_sync(0xffffffffu, code & 1);
    const uint32_t b1 = __ballot_sync(0xffffffffu, (code >> 1) & 1);
    if (lane == 0) codes[(c * Np + k) * 2 + h] = spread_bits(b0) | (spread_bits(b1) << 1);
  }
}

__global__ void __launch_bounds__(kPackWarps * 32)
codes_kernel(const int8_t *__restrict__ geno, int64_t ldg, int N, int Np,
             const int64_t *__restrict__ snp_list, int64_t snp_begin, int64_t n_snps,
             int64_t n_halves, uint64_t *__restrict__ codes) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t hw = (int64_t)blockIdx.x * kPackWarps + warp;  // chunk * 2 + half
  if (hw >= n_halves) return;
  codes_half(geno, ldg, N, Np, snp_list, snp_begin, n_snps, hw, codes, lane);
}

// The same for all SNP sets of a call that have codes (one warp per flattened half).
__global__ void __launch_bounds__(kPackWarps * 32)
codes_batch_kernel(const PackJob *__restrict__ jobs, int n_jobs, int64_t total_halves) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t x = (int64_t)blockIdx.x * kPackWarps + warp;
  if (x >= total_halves) return;
  const PackJob &J = jobs[find_job(jobs, n_jobs, x, true)];
  if (J.codes == nullptr || J.coef_nan) return;  // (such jobs span no halves)
  codes_half(J.geno, J.ldg, J.N, J.Np, J.snp_list, J.snp_begin, J.n_snps, x - J.half0, J.codes,
             lane);
}

// Markers with codes 0..4: one warp per packed SNP slot j of a 32-SNP chunk;
// rows 32i + jj (i = 0..3) of chunk j / 32 get I_i, the metadata the group
// sizes and coefficients (1 / N_i) / h_df (group 4's weighs (D_0+..+D_3)^2).
__global__ void __launch_bounds__(kPackWarps * 32)
pack_multi_kernel(const int8_t *__restrict__ geno, int64_t ldg, int N, int Np,
                  const int64_t *__restrict__ snp_list, int64_t snp_begin, int64_t n_snps,
                  int64_t n_slots, float rh1, float rh2, float rh3, float rh4, int allow_missing,
                  __half *__restrict__ B, ChunkMetaM *__restrict__ meta, unsigned int *status) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t j = (int64_t)blockIdx.x * kPackWarps + warp;
  if (j >= n_slots) return;
  const int64_t c = j / kChunkSnpsM;
  const int jj = (int)(j % kChunkSnpsM);
  __half *rows[kMaxCodeM];
#pragma unroll
  for (int i = 0; i < kMaxCodeM; ++i) rows[i] = B + (c * kChunkRows + kChunkSnpsM * i + jj) * Np;
  ChunkMetaM &m = meta[c];
  const __half one = __int2half_rn(1), zero = __int2half_rn(0);
  const int64_t s = j < n_snps ? (snp_list ? snp_list[j] : snp_begin + j) : -1;
  const int8_t *g = s >= 0 ? geno + s * ldg : nullptr;
  int cnt[kMaxCodeM + 1] = {0, 0, 0, 0, 0};
  bool miss = false, bad = false;
  for (int k = lane; k < Np; k += 32) {
    const int code = (g != nullptr && k < N) ? (int)g[k] : -1;
#pragma unroll
    for (int i = 0; i < kMaxCodeM; ++i) rows[i][k] = code == i ? one : zero;
#pragma unroll
    for (int i = 0; i <= kMaxCodeM; ++i) cnt[i] += code == i;
    if (g != nullptr && k < N) {
      miss |= code == -1;
      bad |= (code < -1 || code > kMaxCodeM);
    }
  }
#pragma unroll
  for (int i = 0; i <= kMaxCodeM; ++i)
    for (int o = 16; o > 0; o >>= 1) cnt[i] += __shfl_xor_sync(0xffffffffu, cnt[i], o);
  miss = __any_sync(0xffffffffu, miss);
  bad = __any_sync(0xffffffffu, bad);
  if (lane == 0) {
    if (bad) atomicOr(status, kDevBadCode);
    if (miss && !allow_missing) atomicOr(status, kDevMissing);
    int groups = 0;
#pragma unroll
    for (int i = 0; i <= kMaxCodeM; ++i) groups += cnt[i] > 0;
    const int df = groups > 0 ? groups - 1 : 0;
    const bool excluded = g == nullptr || (miss && !allow_missing);
    const float rh = df == 1 ? rh1 : df == 2 ? rh2 : df == 3 ? rh3 : rh4;
#pragma unroll
    for (int i = 0; i <= kMaxCodeM; ++i) {
      m.coef[i][jj] = (df > 0 && !excluded && cnt[i] > 0) ? rh / (float)cnt[i] : 0.f;
      m.n[i][jj] = (uint16_t)cnt[i];
    }
    m.snp[jj] = excluded ? -1 : (int32_t)s;
    m.df[jj] = (uint8_t)df;
  }
}
}  // namespace

cudaError_t launch_pack_multi(const int8_t *geno, int64_t ldg, int N, int Np,
                              const int64_t *snp_list, int64_t snp_begin, int64_t n_snps,
                              const double *h, int allow_missing, __half *B, ChunkMetaM *meta,
                              unsigned int *status, cudaStream_t s) {
  const int64_t nchunks = (n_snps + kChunkSnpsM - 1) / kChunkSnpsM;
  const int64_t n_slots = nchunks * kChunkSnpsM;
  if (n_slots == 0) return cudaSuccess;
  const int64_t grid = (n_slots + kPackWarps - 1) / kPackWarps;
  pack_multi_kernel<<<(unsigned)grid, kPackWarps * 32, 0, s>>>(
      geno, ldg, N, Np, snp_list, snp_begin, n_snps, n_slots, (float)(1.0 / h[0]),
      (float)(1.0 / h[1]), (float)(1.0 / h[2]), (float)(1.0 / h[3]), allow_missing, B, meta,
      status);
  return cudaGetLastError();
}

// Packing for the dosage regression of the parametric comparison: the same
// indicators, coefficients rl (2 S_0 + S_1)^2 / S_gg (rl = 1 / ((K-1) r_c^2)).
cudaError_t launch_pack_linear(const int8_t *geno, int64_t ldg, int N, int Np, int64_t snp_begin,
                               int64_t n_snps, double rl, __half *B, ChunkMeta *meta,
                               unsigned int *status, cudaStream_t s) {
  const int64_t nchunks = (n_snps + kChunkSnps - 1) / kChunkSnps;
  const int64_t n_slots = nchunks * kChunkSnps;
  if (n_slots == 0) return cudaSuccess;
  const int64_t grid = (n_slots + kPackWarps - 1) / kPackWarps;
  pack_kernel<<<(unsigned)grid, kPackWarps * 32, 0, s>>>(geno, ldg, N, Np, nullptr, snp_begin, n_snps,
                                                         n_slots, 0, 0.f, 0.f, 0, 0, B, meta, status,
                                                         1, (float)rl);
  return cudaGetLastError();
}

cudaError_t launch_missing_scan(const int8_t *geno, int64_t ldg, int N, int64_t snp_begin,
                                int64_t n_snps, int max_code, unsigned int *n_missing,
                                int64_t *miss_idx, uint64_t *miss_mask, unsigned int *status,
                                uint32_t *flags, cudaStream_t s) {
  if (n_snps <= 0) return cudaSuccess;
  if (flags != nullptr && ldg == N) {  // rows back to back: the flat pre-pass
    cudaError_t e = cudaMemsetAsync(flags, 0, (size_t)((n_snps + 31) / 32) * 4, s);
    if (e != cudaSuccess) return e;
    const int64_t nbytes = n_snps * (int64_t)N;
    const int64_t words = nbytes / 16 + 32;
    const int64_t blocks = std::min<int64_t>((words + 255) / 256, 152 * 16);
    missing_flag_kernel<<<(unsigned)blocks, 256, 0, s>>>(geno + snp_begin * ldg, nbytes, N,
                                                         max_code, flags, status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t fw = (n_snps + 31) / 32;
    missing_collect_kernel<<<(unsigned)((fw + 7) / 8), 256, 0, s>>>(geno, ldg, N, snp_begin, n_snps,
                                                                   flags, n_missing, miss_idx,
                                                                   miss_mask);
    return cudaGetLastError();
  }
  const int64_t grid = (n_snps + kPackWarps - 1) / kPackWarps;
  missing_scan_kernel<<<(unsigned)grid, kPackWarps * 32, 0, s>>>(geno, ldg, N, snp_begin, n_snps,
                                                                 max_code, n_missing, miss_idx,
                                                                 miss_mask, status);
  return cudaGetLastError();
}

cudaError_t launch_pack2(const int8_t *geno, int64_t ldg, int N, int Np, const int64_t *snp_list,
                         int64_t snp_begin, int64_t n_snps, int64_t snp_out_base, double h1,
                         double h2, int allow_missing, int signed_df1, __half *B,
                         ChunkMeta *meta, uint64_t *codes, unsigned int *status, cudaStream_t s) {
  const int64_t nchunks = (n_snps + kChunkSnps - 1) / kChunkSnps;
  const int64_t n_slots = nchunks * kChunkSnps;
  if (n_slots == 0) return cudaSuccess;
  const int64_t grid = (n_slots + kPackWarps - 1) / kPackWarps;
  pack_kernel<<<(unsigned)grid, kPackWarps * 32, 0, s>>>(geno, ldg, N, Np, snp_list, snp_begin,
                                                         n_snps, n_slots, snp_out_base,
                                                         (float)(1.0 / h1), (float)(1.0 / h2),
                                                         allow_missing, signed_df1, B, meta, status,
                                                         0, 0.f);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || codes == nullptr) return e;
  const int64_t n_halves = nchunks * 2;
  const int64_t grid2 = (n_halves + kPackWarps - 1) / kPackWarps;
  codes_kernel<<<(unsigned)grid2, kPackWarps * 32, 0, s>>>(geno, ldg, N, Np, snp_list, snp_begin,
                                                           n_snps, n_halves, codes);
  return cudaGetLastError();
}

cudaError_t launch_pack_batch(const PackJob *jobs, int n_jobs, int64_t total_slots,
                              int64_t total_halves, double h1, double h2, int signed_df1,
                              unsigned int *status, cudaStream_t s) {
  if (n_jobs <= 0) return cudaSuccess;
  if (total_slots > 0) {
    const int64_t warps = (total_slots + 31) / 32;
    const int64_t grid = (warps + kPackWarps - 1) / kPackWarps;
    pack_batch_kernel<<<(unsigned)grid, kPackWarps * 32, 0, s>>>(
        jobs, n_jobs, total_slots, (float)(1.0 / h1), (float)(1.0 / h2), signed_df1, status);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (total_halves > 0) {
    const int64_t grid = (total_halves + kPackWarps - 1) / kPackWarps;
    codes_batch_kernel<<<(unsigned)grid, kPackWarps * 32, 0, s>>>(jobs, n_jobs, total_halves);
    return cudaGetLastError();
  }
  return cudaSuccess;
}

cudaError_t launch_pattern_group(const unsigned int *n_missing, const uint64_t *mask,
                                 const int64_t *miss_idx, int64_t n_snps, PatternScratch &w,
                                 unsigned int *status, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(w.tab_hash, 0, (size_t)w.cap * 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(w.tab_rep, 0x7f, (size_t)w.cap * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(w.n_buckets, 0, 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(w.count, 0, (size_t)n_snps * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(w.fill, 0, (size_t)n_snps * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(w.first, 0xff, (size_t)n_snps * 8, s);
  if (e != cudaSuccess) return e;
  const unsigned g1 = (unsigned)std::min<int64_t>((n_snps + 255) / 256, 152 * 8);
  const unsigned g2 = (unsigned)std::min<int64_t>((w.cap + 255) / 256, 152 * 8);
  pattern_insert_kernel<<<g1, 256, 0, s>>>(n_missing, mask, w.tab_hash, w.tab_rep, w.cap, w.slot_of);
  pattern_number_kernel<<<g2, 256, 0, s>>>(w.tab_hash, w.tab_rep, w.cap, w.tab_id, w.n_buckets, mask,
                                           w.bucket_mask);
  pattern_count_kernel<<<g1, 256, 0, s>>>(n_missing, w.slot_of, w.tab_id, mask, w.bucket_mask,
                                          miss_idx, w.bucket_of, w.count, w.first, status);
  return cudaGetLastError();
}

cudaError_t launch_pattern_lists(const unsigned int *n_missing, const int64_t *miss_idx,
                                 const uint32_t *flags, bool flags_ready, int64_t snp_begin,
                                 int64_t n_snps, PatternScratch &w, int64_t *bucket_list,
                                 int64_t *complete_list, cudaStream_t s) {
  const unsigned g1 = (unsigned)std::min<int64_t>((n_snps + 255) / 256, 152 * 8);
  const int64_t nw = (n_snps + 31) / 32;
  uint32_t *fl = const_cast<uint32_t *>(flags);
  if (!flags_ready) {
    cudaError_t e = cudaMemsetAsync(fl, 0, (size_t)nw * 4, s);
    if (e != cudaSuccess) return e;
    flags_from_idx_kernel<<<g1, 256, 0, s>>>(n_missing, miss_idx, snp_begin, fl);
  }
  pattern_scatter_kernel<<<g1, 256, 0, s>>>(n_missing, w.bucket_of, w.offset, miss_idx, w.fill,
                                            bucket_list);
  complete_offsets_kernel<<<1, 1024, 0, s>>>(flags, n_snps, w.woff);
  complete_scatter_kernel<<<(unsigned)std::min<int64_t>((nw + 255) / 256, 152 * 8), 256, 0, s>>>(
      flags, w.woff, snp_begin, n_snps, complete_list);
  return cudaGetLastError();
}

}  // namespace krux
