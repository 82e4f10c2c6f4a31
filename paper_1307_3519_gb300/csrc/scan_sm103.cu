// scan_sm103.cu -- fused Kruskal-Wallis scan for sm_103a (tcgen05 + TMA + TMEM).
//
// For a tile of 128 traits and a chunk of 64 SNPs the tensor cores contract the
// centred rank matrix A (traits x samples, FP16 integers) with the packed
// indicator rows [I_0 | I_1] of the chunk (Eq. 4: S_i = R I_i^T, here in centred
// form D_i = 2 S_i - N_i (K+1)), accumulating exact FP32 integers in TMEM.  The
// epilogue never writes the rank sums to memory: it evaluates Eq. 2 in centred
// form, H = 3/(K(K+1)C) sum_i D_i^2/N_i with D_2 = -D_0 - D_1 and the tie factor
// C (section "Handling tied data"), compares it with the chi-square threshold of
// the SNP's degrees of freedom (section "P-value calculation and empirical FDR
// correction"), decides pairs within a relative margin of the threshold in
// FP64, and appends hits with one atomic per warp.
//
// Roles (576 threads, one CTA per SM, persistent over work items):
//   warps 0-15: epilogue; warp w reads TMEM lanes 32*(w%4).. (traits) and the
//               16 SNPs 16*(w/4).. of each 64-SNP chunk
//   warp 16   : TMA producer (A tiles stream through nA stages; a B tile of nc
//               chunks stays resident while all trait tiles pass)
//   warp 17   : TMEM allocator and tcgen05.mma issuer (one thread)
// Every mbarrier wait is bounded: on timeout the kernel raises an error bit,
// drains its own asynchronous copies and MMAs, frees TMEM and returns.
#include <atomic>
#include <type_traits>

#include "common.cuh"

namespace krux {

namespace {

// tcgen05 instruction descriptor, kind::f16: D = F32, A = B = F16, both K-major,
// N = 128 (bits 17-22 hold N >> 3), M = 128 (bits 24-28 hold M >> 4).
constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(128 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
// Same with N = 256: one MMA over a pair of chunks whose B rows are interleaved
// per K atom (256 rows of 32 B), writing two adjacent 128-column accumulators.
constexpr uint32_t kIdesc256 = (1u << 4) | ((uint32_t)(256 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
// Two K-major shared-memory layouts: 128-byte swizzle with 64-element K atoms
// (K padded to a multiple of 64, zero-filled by TMA), or 32-byte swizzle with
// 16-element atoms (K padded to a multiple of 16 only).  An atom block holds 128
// rows.
__device__ __forceinline__ uint32_t atom_k(int layout) { return layout ? 16u : 64u; }
__device__ __forceinline__ uint32_t atom_bytes(int layout) { return layout ? 4096u : 16384u; }
// byte offset of K step k (16 elements) inside a tile
__device__ __forceinline__ uint32_t kstep_off(int layout, int k) {
  return layout ? (uint32_t)k * 4096u : (uint32_t)(k >> 2) * 16384u + (uint32_t)(k & 3) * 32u;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor of a K-major swizzled tile: start address,
// leading offset (unused for these layouts), 8-row group stride (SBO: 1024 B for
// the 128-byte swizzle, 256 B for the 32-byte swizzle), version 1, layout type
// (2 = 128-byte swizzle, 6 = 32-byte swizzle).
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, int layout) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;
  d |= (uint64_t)((layout ? 256u : 1024u) >> 4) << 32;
  d |= (uint64_t)1u << 46;
  d |= (uint64_t)(layout ? 6u : 2u) << 61;
  return d;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0u;
}
// The same with a suspend-time hint: a thread whose phase is not complete sleeps
// (issuing nothing) until the phase completes or about `ns` nanoseconds pass.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint32_t bar, uint32_t parity, uint32_t ns) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(ns)
      : "memory");
  return ok != 0u;
}
// Suspend hint of the bounded waits (ns): long enough that a waiting thread
// takes no issue slots from the working warps of its scheduler, short enough
// that timeouts and aborts are still noticed promptly.
constexpr uint32_t kWaitSleepNs = 200000u;

struct WaitCtl {
  volatile int *abort_flag;
  unsigned int *status;
  long long limit;
};

// Bounded wait for the phase of parity `parity`; false on timeout or abort.
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity, const WaitCtl &w,
                                      unsigned int where) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (mbar_try_wait_sleep(bar, parity, kWaitSleepNs)) return true;
    if (*w.abort_flag) return false;
    if (clock64() - t0 > w.limit) {
      *w.abort_flag = 1;
      atomicOr(w.status, kDevTimeout);
      atomicMax(w.status + 1, where);
      return false;
    }
  }
}

// The same bounded wait, reading its limit and status words from the kernel
// parameters and the abort flag through its shared-memory address (keeps no
// per-thread copies of them in registers).
__device__ __forceinline__ bool wait_bar_p(uint32_t bar, uint32_t parity, const ScanParams &p,
                                         uint32_t abort_addr, unsigned int where) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (mbar_try_wait_sleep(bar, parity, kWaitSleepNs)) return true;
    int ab;
    asm volatile("ld.volatile.shared.u32 %0, [%1];" : "=r"(ab) : "r"(abort_addr) : "memory");
    if (ab) return false;
    if (clock64() - t0 > p.timeout_cycles) {
      asm volatile("st.volatile.shared.u32 [%0], %1;" ::"r"(abort_addr), "r"(1) : "memory");
      atomicOr(p.status, kDevTimeout);
      atomicMax(p.status + 1, where);
      return false;
    }
  }
}

// Wait used while shutting down: ignores the abort flag (copies and MMAs already
// issued must land before the CTA can release its shared memory and TMEM) and
// gives up only after a fixed bound of about two seconds.
// (inline: it is also reached by warps that have given registers away with
// setmaxnreg, which must call no function compiled for more registers)
__device__ __forceinline__ void wait_drain(uint32_t bar, uint32_t parity, unsigned int *status,
                                           unsigned int where) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > 4000000000LL) {
      atomicOr(status, kDevTimeout);
      atomicMax(status + 1, where);
      return;
    }
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
      "%3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes,
                                          uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void prefetch_map(const CUtensorMap *map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t da, uint64_t db, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

#define KRUX_LD16_REGS(r)                                                                       \
  "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),          \
      "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),  \
      "=r"(r[14]), "=r"(r[15])

// 16 consecutive fp32 columns of this warp's 32 TMEM lanes (one lane per thread).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[kEpiSnps]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];"
      : KRUX_LD16_REGS(r)
      : "r"(taddr)
      : "memory");
}
// 8 consecutive fp32 columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[kEpiSnpsM]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Same quadratic form without the bound; with permutation batches the df-1 SNPs
// carry negated alpha, gamma so the sign of the result tells the df apart.
__device__ __forceinline__ float kw_s(float u, float v, float al, float be, float ga) {
  const float w = fmaf(be, v, u);
  const float e = ga * v;
  const float t = e * v;
  const float f = al * w;
  return fmaf(f, w, t);
}

// -ln p for df = 1: -ln erfc(x) = x^2 - ln erfcx(x), x = sqrt(H/2) (no underflow).
__device__ __forceinline__ float key1f(float H) {
  const float x2 = 0.5f * H;
  if (!(x2 > 0.f)) return 0.f;
  return x2 - logf(erfcxf(sqrtf(x2)));
}
__device__ __forceinline__ double key64_of(double H, int df) {
  if (df == 2) return 0.5 * H;
  if (df == 1) {
    const double x2 = 0.5 * H;
    if (!(x2 > 0.0)) return 0.0;
    return x2 - log(erfcx(sqrt(x2)));
  }
  return 0.0;
}

// cis mode: only pairs whose SNP and trait lie within the window are reported.
__device__ __forceinline__ bool in_cis_window(const ScanParams &p, int snp, int trait) {
  if (p.cis_window < 0) return true;
  const long long d = (long long)(p.cis_snp_pos[snp] - p.cis_trait_pos[trait]);
  return d <= p.cis_window && -d <= p.cis_window;
}

// FDR histogram bin of a pair with -ln p = key: b = floor((-log10 p - l0) / w),
// clamped to [0, bins).
__device__ __forceinline__ int fdr_bin(double key, double l0, double w, int bins) {
  const double x = (key * 0.43429448190325182765 - l0) / w;
  if (!(x >= 1.0)) return 0;
  if (x >= (double)(bins - 1)) return bins - 1;
  return (int)x;
}

// Upper chi-square tail with df = 1..4 degrees of freedom, Q(df/2, H/2) for
// integer and half-integer shape: df 1: erfc(sqrt x); df 2: e^-x;
// df 3: erfc(sqrt x) + 2 sqrt(x / pi) e^-x; df 4: e^-x (1 + x); x = H/2.
__device__ __forceinline__ double chi2_tail64(double H, int df) {
  if (df <= 0 || !(H > 0.0)) return 1.0;
  const double x = 0.5 * H;
  if (df == 1) return erfc(sqrt(x));
  if (df == 2) return exp(-x);
  if (df == 3) return erfc(sqrt(x)) + 1.12837916709551257390 * sqrt(x) * exp(-x);
  return exp(-x) * (1.0 + x);
}

// p-value of the pair in FP64 from the exact centred sums and group sizes.
__device__ __forceinline__ double kw_p64(double H, int df) {
  if (df == 1) return erfc(sqrt(0.5 * H));
  if (df == 2) return exp(-0.5 * H);
  return 1.0;
}
// The reported p of a hit (df 1, 2; the decisions use kw_p64): exp(-x), x = H/2, as
// 2^-k 2^-f with k = floor(x log2 e) and f the fraction, both from FP64, and 2^-f
// from exp2f; for df = 1, erfc(z) = exp(-z^2) erfcx(z), z = sqrt(x), with erfcx in
// FP32 (smooth, so its argument's rounding barely moves it).  Relative error a few
// 1e-7; no FP64 transcendental.
__device__ __forceinline__ double kw_p_report(double H, int df) {
  const double x = 0.5 * H;
  if (!(x > 0.0)) return 1.0;
  const double t = x * 1.4426950408889634074;  // x log2(e)
  const double k = floor(t);
  if (k > 1000.0) return 0.0;
  const double two_mk = __longlong_as_double((long long)(1023 - (int)k) << 52);  // 2^-k
  double e = (double)exp2f(-(float)(t - k)) * two_mk;
  if (df == 1) e *= (double)erfcxf(sqrtf((float)x));
  return e;
}
__device__ __forceinline__ double kw_H64(int u, int v, int n0, int n1, int n2, double cfac) {
  const double D0 = (double)u, D1 = (double)v, D2 = -(double)(u + v);
  double Q = 0.0;
  if (n0 > 0) Q += D0 * D0 / (double)n0;
  if (n1 > 0) Q += D1 * D1 / (double)n1;
  if (n2 > 0) Q += D2 * D2 / (double)n2;
  return cfac * Q;
}

struct EpiTrait {
  int trait;        // global trait row of this thread (may be >= T in the last tile)
  bool valid;
  float ntlo, nthi; // -tau (1 -/+ margin)
  double cfac;
  int nan_cnt;      // 0 unless the rank set has NaN in this trait
  const uint16_t *nan_idx;
};

// Group sizes of a pair after removing the trait's NaN samples (section
// "Handling missing values": N_i(n,m) counts the samples present for both).
__device__ __forceinline__ void pair_counts(int nan_cnt, const uint16_t *nan_idx,
                                            const ChunkMeta &m, const uint64_t *codes, int jj,
                                            int &n0, int &n1, int &n2) {
  n0 = m.n[0][jj];
  n1 = m.n[1][jj];
  n2 = m.n[2][jj];
  for (int i = 0; i < nan_cnt; ++i) {
    const int k = nan_idx[i];
    const int code = (int)((codes[k * 2 + (jj >> 5)] >> (2 * (jj & 31))) & 3ull);
    n0 -= code == 0;
    n1 -= code == 1;
    n2 -= code == 2;
  }
}

__device__ __forceinline__ int df_of(int n0, int n1, int n2) {
  const int g = (n0 > 0) + (n1 > 0) + (n2 > 0);
  return g > 0 ? g - 1 : 0;
}

// ---- packed fp32x2 helpers (two SNPs per instruction) ----------------------
__device__ __forceinline__ uint64_t pk2(uint32_t a, uint32_t b) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "r"(a), "r"(b));
  return r;
}
__device__ __forceinline__ void upk2(uint64_t r, uint32_t &a, uint32_t &b) {
  asm("mov.b64 {%0, %1}, %2;" : "=r"(a), "=r"(b) : "l"(r));
}
__device__ __forceinline__ uint64_t ffma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ uint64_t fmul2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t fadd2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ float fmax3(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
__device__ __forceinline__ float fmin3(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// Hot test of kEpiSnps SNPs: true when some pair may lie at or above the lower edge of
// the band (q >= 0).  Two SNPs per packed instruction:
//   w = u + beta v,  q = alpha w^2 + gamma v^2 - tau (1 - margin)
// (with permutation batches the form is signed by df and |form| is tested).
template <bool kSigned>
__device__ __forceinline__ bool hit_fast(const uint32_t (&d0)[kEpiSnps], const uint32_t (&d1)[kEpiSnps],
                                         const ChunkMeta &m, int h, float ntlo) {
  const uint64_t *al = reinterpret_cast<const uint64_t *>(m.alpha + kEpiSnps * h);
  const uint64_t *be = reinterpret_cast<const uint64_t *>(m.beta + kEpiSnps * h);
  const uint64_t *ga = reinterpret_cast<const uint64_t *>(m.gamma + kEpiSnps * h);
  const uint64_t nt2 = pk2(__float_as_uint(ntlo), __float_as_uint(ntlo));
  uint32_t acc = 0xffffffffu;
#pragma unroll
  for (int j = 0; j < kEpiSnps / 2; j += 2) {
    const ulonglong2 A = *reinterpret_cast<const ulonglong2 *>(al + j);
    const ulonglong2 B = *reinterpret_cast<const ulonglong2 *>(be + j);
    const ulonglong2 G = *reinterpret_cast<const ulonglong2 *>(ga + j);
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int jj = 2 * (j + t);
      const uint64_t u2 = pk2(d0[jj], d0[jj + 1]);
      const uint64_t v2 = pk2(d1[jj], d1[jj + 1]);
      const uint64_t a2 = t ? A.y : A.x, b2 = t ? B.y : B.x, g2 = t ? G.y : G.x;
      const uint64_t w2 = ffma2(b2, v2, u2);
      const uint64_t e2 = fmul2(g2, v2);
      uint64_t q2;
      if (!kSigned) {
        q2 = ffma2(e2, v2, nt2);
        q2 = ffma2(fmul2(a2, w2), w2, q2);
      } else {
        q2 = ffma2(fmul2(a2, w2), w2, fmul2(e2, v2));
        q2 = fadd2(q2 & 0x7fffffff7fffffffull, nt2);
      }
      uint32_t qa, qb;
      upk2(q2, qa, qb);
      acc &= qa & qb;
    }
  }
  return (int)acc >= 0;
}

// Small non-negative integer (< 2^23) to float, exactly, without a conversion
// instruction: the integer sits in the mantissa of 2^23.
__device__ __forceinline__ float small_int_f(int x) {
  return __int_as_float(0x4b000000 | x) - 8388608.f;
}

// Hot test of a chunk half for a trait with NaN samples (section "Handling missing
// values": N_i(n,m) counts the samples present for both).  Each pair's group sizes
// come from the genotype codes of the trait's c NaN samples: k_i = the NaN samples
// with genotype i, summed over the samples in 4-bit fields (c <= 15; more take the
// rare path at once), n_i' = n_i - k_i.  The test sum_i D_i^2 / n_i' >= q_df is
// taken without a division, as u^2 n1 n2 + v^2 n0 n2 + w^2 n0 n1 >= q_df n0 n1 n2
// (an emptied group has D_i = 0 and counts as n_i' = 1; q_df of the pair's own df,
// q1, q2 = h_df (1 - margin) / cfac).  True if some pair may be a hit; the rare
// path decides it exactly.
__device__ __forceinline__ bool hit_fast_nan(const uint32_t (&d0)[kEpiSnps],
                                             const uint32_t (&d1)[kEpiSnps], const ChunkMeta &m,
                                             int h, const uint64_t *codes, int c,
                                             const uint16_t *nan_idx, float q1, float q2) {
  if (c > 15) return true;
  // k_i of SNPs 8 b .. 8 b + 7 in the 4-bit fields of kb[i][b]
  uint32_t kb[3][2] = {{0u, 0u}, {0u, 0u}, {0u, 0u}};
  for (int i = 0; i < c; ++i) {
    const int k = nan_idx[i];
    const uint32_t x = (uint32_t)(codes[k * 2 + (h >> 1)] >> (32 * (h & 1)));
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      // the 8 two-bit codes of this half-word, each moved to a 4-bit field
      uint32_t z = (x >> (16 * b)) & 0xffffu;
      z = (z | (z << 8)) & 0x00ff00ffu;
      z = (z | (z << 4)) & 0x0f0f0f0fu;
      z = (z | (z << 2)) & 0x33333333u;
      const uint32_t lo = z & 0x11111111u, hi = (z >> 1) & 0x11111111u;
      kb[0][b] += ~(lo | hi) & 0x11111111u;
      kb[1][b] += lo & ~hi;
      kb[2][b] += hi & ~lo;
    }
  }
  const int jb = kEpiSnps * h;
  const uint4 *p0 = reinterpret_cast<const uint4 *>(&m.n[0][jb]);
  const uint4 *p1 = reinterpret_cast<const uint4 *>(&m.n[1][jb]);
  const uint4 *p2 = reinterpret_cast<const uint4 *>(&m.n[2][jb]);
  const float inf = __int_as_float(0x7f800000);
  bool need = false;
#pragma unroll
  for (int hb = 0; hb < 2; ++hb) {  // SNPs 8 hb .. 8 hb + 7
    const uint4 a0 = p0[hb], a1 = p1[hb], a2 = p2[hb];
    const uint32_t w0[4] = {a0.x, a0.y, a0.z, a0.w}, w1[4] = {a1.x, a1.y, a1.z, a1.w},
                   w2[4] = {a2.x, a2.y, a2.z, a2.w};
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int j = 8 * hb + t;
      const int sh = (t & 1) * 16;
      const int n0 = (int)((w0[t >> 1] >> sh) & 0xffffu) - (int)((kb[0][hb] >> (4 * t)) & 15u);
      const int n1 = (int)((w1[t >> 1] >> sh) & 0xffffu) - (int)((kb[1][hb] >> (4 * t)) & 15u);
      const int n2 = (int)((w2[t >> 1] >> sh) & 0xffffu) - (int)((kb[2][hb] >> (4 * t)) & 15u);
      const int groups = (n0 > 0) + (n1 > 0) + (n2 > 0);
      const float thr = groups == 3 ? q2 : (groups == 2 ? q1 : inf);
      const float f0 = small_int_f(max(n0, 1)), f1 = small_int_f(max(n1, 1)),
                  f2 = small_int_f(max(n2, 1));
      const float u = __uint_as_float(d0[j]), v = __uint_as_float(d1[j]);
      const float w = -(u + v);
      const float f12 = f1 * f2;
      const float num = fmaf(w * w, f0 * f1, fmaf(v * v, f0 * f2, u * u * f12));
      need |= fmaf(-thr, f0 * f12, num) >= 0.f;
    }
  }
  return need;
}

// Rare path of a hit-mode chunk half: dense FP64 output, traits with NaN,
// classification of candidates (FP64 inside the band) and the warp-aggregated
// append of hits.  Called by the whole warp; `dv` holds this lane's kEpiSnps D_0
// then kEpiSnps D_1 values (a local copy, so the hot path keeps them in registers).
__device__ __noinline__ void hit_slow(const uint32_t *dv, bool mine, const ChunkMeta &m,
                                      const uint64_t *codes, int h, int trait, bool valid,
                                      float ntlo, float nthi, double cfac, int nan_cnt,
                                      const uint16_t *nan_idx, const GroupDesc &g,
                                      const ScanParams &p, int lane) {
  const int jb = kEpiSnps * h;
  uint32_t hitmask = 0;
  if (mine && valid) {
    const float *al = m.alpha + jb, *be = m.beta + jb, *ga = m.gamma + jb;
    for (int j = 0; j < kEpiSnps; ++j) {
      const int snp = m.snp[jb + j];
      if (snp < 0 || !in_cis_window(p, snp, trait)) continue;
      const float u = __uint_as_float(dv[j]), v = __uint_as_float(dv[kEpiSnps + j]);
      if (p.dense || nan_cnt > 0) {
        int n0, n1, n2;
        pair_counts(nan_cnt, nan_idx, m, codes, jb + j, n0, n1, n2);
        const int df = df_of(n0, n1, n2);
        if (p.dense) {
          const double H = (df > 0 && cfac > 0.0) ? kw_H64((int)u, (int)v, n0, n1, n2, cfac) : 0.0;
          const double pv = (df > 0 && cfac > 0.0) ? kw_p64(H, df) : 1.0;
          const int64_t o = (int64_t)trait * g.dense_ld + (snp - g.dense_snp0);
          g.dense_H[o] = H;
          g.dense_p[o] = pv;
          if (pv < p.pthresh) hitmask |= 1u << j;
        } else if (df > 0) {
          const float w = -(u + v);
          float Q = 0.f;
          if (n0 > 0) Q += u * u / (float)n0;
          if (n1 > 0) Q += v * v / (float)n1;
          if (n2 > 0) Q += w * w / (float)n2;
          const float hq = (float)cfac * Q;
          const float hd = df == 1 ? p.h1 : p.h2;
          if (hq > hd * (1.f - p.margin)) {
            bool hit = hq > hd * (1.f + p.margin);
            if (!hit) hit = kw_p64(kw_H64((int)u, (int)v, n0, n1, n2, cfac), df) < p.pthresh;
            if (hit) hitmask |= 1u << j;
          }
        }
      } else {
        float sv = kw_s(u, v, al[j], be[j], ga[j]);
        if (p.signed_coef) sv = fabsf(sv);
        if (sv + ntlo >= 0.f) {
          bool hit = sv + nthi > 0.f;
          if (!hit) {
            const double H = kw_H64((int)u, (int)v, m.n[0][jb + j], m.n[1][jb + j], m.n[2][jb + j], cfac);
            hit = kw_p64(H, m.df[jb + j]) < p.pthresh;
          }
          if (hit) hitmask |= 1u << j;
        }
      }
    }
  }
  if (!__any_sync(0xffffffffu, hitmask != 0u)) return;
  // warp-aggregated append: one atomic per warp
  const int cnt = __popc(hitmask);
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(g.counter, (unsigned long long)total);
  base = __shfl_sync(0xffffffffu, base, 0);
  unsigned long long idx = base + (unsigned long long)(incl - cnt);
  const unsigned long long cap = (unsigned long long)g.capacity;
  while (hitmask) {
    const int j = __ffs(hitmask) - 1;
    hitmask &= hitmask - 1u;
    if (idx < cap) {
      int n0, n1, n2;
      pair_counts(nan_cnt, nan_idx, m, codes, jb + j, n0, n1, n2);
      krux_hit r;
      r.trait = (uint32_t)trait;
      r.snp = (uint32_t)m.snp[jb + j];
      r.d0 = (int32_t)__uint_as_float(dv[j]);
      r.d1 = (int32_t)__uint_as_float(dv[kEpiSnps + j]);
      st_hit(g.hits + idx, r);
      HitAux a;
      a.n0 = (uint16_t)n0;
      a.n1 = (uint16_t)n1;
      a.n2 = (uint16_t)n2;
      a.group = (uint16_t)g.group_id;
      st_aux(g.aux + idx, a);
    }
    ++idx;
  }
}

// FP64 decision for a pair inside the band (rare): p < P_c from the exact sums.
__device__ __noinline__ bool decide64(float u, float v, int n0, int n1, int n2, int df, double cfac,
                                      double pthresh) {
  return kw_p64(kw_H64((int)u, (int)v, n0, n1, n2, cfac), df) < pthresh;
}
// The same decision inline, for the event warps of the plain scan form: they run
// with fewer registers than the kernel was compiled for (setmaxnreg) and must not
// call a function compiled for the full count.
__device__ __forceinline__ bool decide64_inl(float u, float v, int n0, int n1, int n2, int df,
                                             double cfac, double pthresh) {
  return kw_p64(kw_H64((int)u, (int)v, n0, n1, n2, cfac), df) < pthresh;
}


// Rare path of a hit-mode chunk half without dense output or NaN traits, called
// by the whole warp (inlined: a call costs more in register saves than the
// extra code costs the hot loop).  Each lane classifies its candidates (two SNPs per packed
// instruction: at or above the upper band edge -> hit, inside the band -> FP64),
// then the warp appends the hits in lane order with every lane writing records
// (the source lane of record r is the first lane with inclusive count > r, found
// by a binary search over shuffles; its SNP is the (r - excl)-th set bit of that
// lane's mask and the sums come by shuffle), so the records of an event whose
// hits sit in one lane still leave in whole vector stores.  Records first fill this warp's own
// staging segment (`wn` records already there; no atomic); whatever does not fit
// goes straight to the caller's list through the global counter.  Returns the
// number of hits found (the warp's segment counter advances by it).  A compaction
// pass appends the segments after the launch.
__device__ __forceinline__ unsigned int hit_event(const uint32_t *dv, bool mine, const ChunkMeta &m,
                                               int h, int trait, float ntlo, float nthi,
                                               double cfac, const GroupDesc &g,
                                               const ScanParams &p, unsigned int wn, int lane) {
  const int jb = kEpiSnps * h;
  uint32_t hm = 0;
  if (mine) {
    const uint64_t *al = reinterpret_cast<const uint64_t *>(m.alpha + jb);
    const uint64_t *be = reinterpret_cast<const uint64_t *>(m.beta + jb);
    const uint64_t *ga = reinterpret_cast<const uint64_t *>(m.gamma + jb);
    const uint64_t lo2c = pk2(__float_as_uint(ntlo), __float_as_uint(ntlo));
    const uint64_t hi2c = pk2(__float_as_uint(nthi), __float_as_uint(nthi));
    uint32_t below = 0, not_sure = 0;  // sign bits of s - tau(1 -/+ margin)
#pragma unroll
    for (int j = 0; j < kEpiSnps; j += 2) {
      const uint64_t u2 = pk2(dv[j], dv[j + 1]);
      const uint64_t v2 = pk2(dv[kEpiSnps + j], dv[kEpiSnps + j + 1]);
      const uint64_t w2 = ffma2(be[j / 2], v2, u2);
      const uint64_t e2 = fmul2(ga[j / 2], v2);
      uint64_t s2 = ffma2(fmul2(al[j / 2], w2), w2, fmul2(e2, v2));
      if (p.signed_coef) s2 &= 0x7fffffff7fffffffull;
      uint32_t la, lb, ha, hb;
      upk2(fadd2(s2, lo2c), la, lb);
      upk2(fadd2(s2, hi2c), ha, hb);
      below |= ((la >> 31) | ((lb >> 31) << 1)) << j;
      not_sure |= ((ha >> 31) | ((hb >> 31) << 1)) << j;
    }
    uint32_t cand = ~below & ((1u << kEpiSnps) - 1u);
    if (p.cis_window < 0) {
      // padding and excluded SNPs carry zero coefficients and are never candidates:
      // the clear hits need no loop, only the band goes on to FP64
      hm = p.provisional != 0 ? cand : (cand & ~not_sure);
      cand = p.provisional != 0 ? 0u : (cand & not_sure);
    }
    while (cand) {
      const int j = __ffs(cand) - 1;
      cand &= cand - 1u;
      if (m.snp[jb + j] < 0 || !in_cis_window(p, m.snp[jb + j], trait)) continue;
      bool hit = p.provisional != 0 || ((not_sure >> j) & 1u) == 0u;
      if (!hit)
        hit = decide64(__uint_as_float(dv[j]), __uint_as_float(dv[kEpiSnps + j]), m.n[0][jb + j],
                       m.n[1][jb + j], m.n[2][jb + j], m.df[jb + j], cfac, p.pthresh);
      if (hit) hm |= 1u << j;
    }
  }
  const unsigned int total = __reduce_add_sync(0xffffffffu, (unsigned int)__popc(hm));
  if (total == 0u) return 0u;
  const unsigned int cap = (unsigned int)p.seg_cap;
  const unsigned int sbase = wn;
  const unsigned int over_from = sbase > cap ? sbase : cap;  // first index beyond the segment
  const unsigned int n_over = sbase + total > over_from ? sbase + total - over_from : 0u;
  unsigned long long gbase = 0;
  if (lane == 0 && n_over > 0) gbase = atomicAdd(g.counter, (unsigned long long)n_over);
  gbase = __shfl_sync(0xffffffffu, gbase, 0);
  const size_t seg0 = ((size_t)blockIdx.x * kEpiWarps + (threadIdx.x >> 5)) * cap;
  const uint16_t gid = (uint16_t)g.group_id;
  // lane l's hits take record indices [incl_l - cnt_l, incl_l) after sbase
  const unsigned int cnt = (unsigned int)__popc(hm);
  unsigned int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  for (unsigned int r0 = 0; r0 < total; r0 += 32u) {
    const unsigned int r = r0 + (unsigned int)lane;
    int lo = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {  // first lane with incl > r
      const unsigned int v = __shfl_sync(0xffffffffu, incl, lo + step - 1);
      if (v <= r) lo += step;
    }
    const int src = lo < 31 ? lo : 31;
    const unsigned int src_incl = __shfl_sync(0xffffffffu, incl, src);
    const unsigned int src_cnt = __shfl_sync(0xffffffffu, cnt, src);
    const uint32_t src_hm = __shfl_sync(0xffffffffu, hm, src);
    const uint32_t src_trait = __shfl_sync(0xffffffffu, (uint32_t)trait, src);
    const int j = (int)__fns(src_hm, 0u, (int)(r - (src_incl - src_cnt)) + 1);
    uint32_t du = 0u, dw = 0u;
#pragma unroll
    for (int jj = 0; jj < kEpiSnps; ++jj) {
      const uint32_t a = __shfl_sync(0xffffffffu, dv[jj], src);
      const uint32_t b = __shfl_sync(0xffffffffu, dv[kEpiSnps + jj], src);
      if (jj == j) {
        du = a;
        dw = b;
      }
    }
    if (r < total) {
      const unsigned int idx = sbase + r;
      krux_hit rec;
      rec.trait = src_trait;
      rec.snp = (uint32_t)m.snp[jb + j];
      rec.d0 = (int32_t)__uint_as_float(du);
      rec.d1 = (int32_t)__uint_as_float(dw);
      HitAux x;
      x.n0 = m.n[0][jb + j];
      x.n1 = m.n[1][jb + j];
      x.n2 = m.n[2][jb + j];
      x.group = gid;
      if (idx < cap) {
        st_hit(p.seg_hits + seg0 + idx, rec);
        st_aux(p.seg_aux + seg0 + idx, x);
      } else {
        const unsigned long long gi = gbase + (idx - over_from);
        if (gi < (unsigned long long)g.capacity) {
          st_hit(g.hits + gi, rec);
          st_aux(g.aux + gi, x);
        }
      }
    }
  }
  return total;
}

// The same event with the records appended SNP column by SNP column (lanes with
// a hit of the same SNP take consecutive records).  Smaller than the lane-order
// append above; the permutation form uses it, where register room matters more.
__device__ __forceinline__ unsigned int hit_event_cols(const uint32_t *dv, bool mine, const ChunkMeta &m,
                                               int h, int trait, float ntlo, float nthi,
                                               double cfac, const GroupDesc &g,
                                               const ScanParams &p, unsigned int wn, int lane) {
  const int jb = kEpiSnps * h;
  uint32_t hm = 0;
  if (mine) {
    const uint64_t *al = reinterpret_cast<const uint64_t *>(m.alpha + jb);
    const uint64_t *be = reinterpret_cast<const uint64_t *>(m.beta + jb);
    const uint64_t *ga = reinterpret_cast<const uint64_t *>(m.gamma + jb);
    const uint64_t lo2c = pk2(__float_as_uint(ntlo), __float_as_uint(ntlo));
    const uint64_t hi2c = pk2(__float_as_uint(nthi), __float_as_uint(nthi));
    uint32_t below = 0, not_sure = 0;  // sign bits of s - tau(1 -/+ margin)
#pragma unroll
    for (int j = 0; j < kEpiSnps; j += 2) {
      const uint64_t u2 = pk2(dv[j], dv[j + 1]);
      const uint64_t v2 = pk2(dv[kEpiSnps + j], dv[kEpiSnps + j + 1]);
      const uint64_t w2 = ffma2(be[j / 2], v2, u2);
      const uint64_t e2 = fmul2(ga[j / 2], v2);
      uint64_t s2 = ffma2(fmul2(al[j / 2], w2), w2, fmul2(e2, v2));
      if (p.signed_coef) s2 &= 0x7fffffff7fffffffull;
      uint32_t la, lb, ha, hb;
      upk2(fadd2(s2, lo2c), la, lb);
      upk2(fadd2(s2, hi2c), ha, hb);
      below |= ((la >> 31) | ((lb >> 31) << 1)) << j;
      not_sure |= ((ha >> 31) | ((hb >> 31) << 1)) << j;
    }
    uint32_t cand = ~below & ((1u << kEpiSnps) - 1u);
    while (cand) {
      const int j = __ffs(cand) - 1;
      cand &= cand - 1u;
      if (m.snp[jb + j] < 0 || !in_cis_window(p, m.snp[jb + j], trait)) continue;
      bool hit = p.provisional != 0 || ((not_sure >> j) & 1u) == 0u;
      if (!hit)
        hit = decide64(__uint_as_float(dv[j]), __uint_as_float(dv[kEpiSnps + j]), m.n[0][jb + j],
                       m.n[1][jb + j], m.n[2][jb + j], m.df[jb + j], cfac, p.pthresh);
      if (hit) hm |= 1u << j;
    }
  }
  const unsigned int total = __reduce_add_sync(0xffffffffu, (unsigned int)__popc(hm));
  if (total == 0u) return 0u;
  const unsigned int cap = (unsigned int)p.seg_cap;
  const unsigned int sbase = wn;
  const unsigned int over_from = sbase > cap ? sbase : cap;  // first index beyond the segment
  const unsigned int n_over = sbase + total > over_from ? sbase + total - over_from : 0u;
  unsigned long long gbase = 0;
  if (lane == 0 && n_over > 0) gbase = atomicAdd(g.counter, (unsigned long long)n_over);
  gbase = __shfl_sync(0xffffffffu, gbase, 0);
  const size_t seg0 = ((size_t)blockIdx.x * kEpiWarps + (threadIdx.x >> 5)) * cap;
  const uint32_t below_me = (1u << lane) - 1u;
  const uint16_t gid = (uint16_t)g.group_id;
  unsigned int run = sbase;  // index of the next record (same in every lane)
  uint32_t cols = __reduce_or_sync(0xffffffffu, hm);
  while (cols) {
    const int j = __ffs(cols) - 1;
    cols &= cols - 1u;
    const bool mine_j = (hm >> j) & 1u;
    const uint32_t bal = __ballot_sync(0xffffffffu, mine_j);
    if (mine_j) {
      const unsigned int idx = run + (unsigned int)__popc(bal & below_me);
      krux_hit r;
      r.trait = (uint32_t)trait;
      r.snp = (uint32_t)m.snp[jb + j];
      r.d0 = (int32_t)__uint_as_float(dv[j]);
      r.d1 = (int32_t)__uint_as_float(dv[kEpiSnps + j]);
      HitAux x;
      x.n0 = m.n[0][jb + j];
      x.n1 = m.n[1][jb + j];
      x.n2 = m.n[2][jb + j];
      x.group = gid;
      if (idx < cap) {
        st_hit(p.seg_hits + seg0 + idx, r);
        st_aux(p.seg_aux + seg0 + idx, x);
      } else {
        const unsigned long long gi = gbase + (idx - over_from);
        if (gi < (unsigned long long)g.capacity) {
          st_hit(g.hits + gi, r);
          st_aux(g.aux + gi, x);
        }
      }
    }
    run += (unsigned int)__popc(bal);
  }
  return total;
}

// ---- the plain scan form: one warp per chunk of an accumulator pair ----------
// 16 consecutive fp32 columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_ld16p(uint32_t taddr, uint32_t *r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
// kFastSnps / 2 = 16 SNPs' D_0 and D_1 (columns c and 64 + c of the chunk) of this lane.
__device__ __forceinline__ void tmem_ld_half(uint32_t taddr, uint32_t (&u)[kFastSnps / 2],
                                             uint32_t (&v)[kFastSnps / 2]) {
  tmem_ld16p(taddr, u);
  tmem_ld16p(taddr + 64u, v);
}

// Hot test of kFastSnps SNPs of a chunk (from SNP `off`) for this lane's trait:
// true when some pair may lie at or above the lower edge of the band (q >= 0),
// two SNPs per packed instruction, w = u + beta v, q = alpha w^2 + gamma v^2 -
// tau (1 - margin).  Blocks of 16 SNPs; two sign accumulators.
// The coefficients come from three arrays of a chunk (ChunkMeta's, or a CoefSet).
template <int NS>
__device__ __forceinline__ bool hit_fast_wc(const uint32_t (&d0)[NS], const uint32_t (&d1)[NS],
                                            const float *alpha, const float *beta,
                                            const float *gamma, int off, float ntlo) {
  const uint64_t nt2 = pk2(__float_as_uint(ntlo), __float_as_uint(ntlo));
  uint32_t acc0 = 0xffffffffu, acc1 = 0xffffffffu;  // AND of the sign bits (two chains)
#pragma unroll
  for (int b = 0; b < NS / 16; ++b) {
    const uint64_t *al = reinterpret_cast<const uint64_t *>(alpha + off + 16 * b);
    const uint64_t *be = reinterpret_cast<const uint64_t *>(beta + off + 16 * b);
    const uint64_t *ga = reinterpret_cast<const uint64_t *>(gamma + off + 16 * b);
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
      const ulonglong2 A = *reinterpret_cast<const ulonglong2 *>(al + j);
      const ulonglong2 B = *reinterpret_cast<const ulonglong2 *>(be + j);
      const ulonglong2 G = *reinterpret_cast<const ulonglong2 *>(ga + j);
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int jj = 16 * b + 2 * (j + t);
        const uint64_t u2 = pk2(d0[jj], d0[jj + 1]);
        const uint64_t v2 = pk2(d1[jj], d1[jj + 1]);
        const uint64_t a2 = t ? A.y : A.x, b2 = t ? B.y : B.x, g2 = t ? G.y : G.x;
        const uint64_t w2 = ffma2(b2, v2, u2);
        const uint64_t e2 = fmul2(g2, v2);
        uint64_t q2 = ffma2(e2, v2, nt2);
        q2 = ffma2(fmul2(a2, w2), w2, q2);
        uint32_t qa, qb;
        upk2(q2, qa, qb);
        if (t) acc1 &= qa & qb;
        else acc0 &= qa & qb;
      }
    }
    // compiler barrier: the next block's coefficient loads are not hoisted above
    // this one (the accumulator registers stay live throughout)
    if (b + 1 < NS / 16) asm volatile("" ::: "memory");
  }
  return (int)(acc0 & acc1) >= 0;
}
template <int NS>
__device__ __forceinline__ bool hit_fast_w(const uint32_t (&d0)[NS], const uint32_t (&d1)[NS],
                                           const ChunkMeta &m, int off, float ntlo) {
  return hit_fast_wc<NS>(d0, d1, m.alpha, m.beta, m.gamma, off, ntlo);
}

// Two-sided hot test of a permutation batch, whose df-1 SNPs carry a negated form
// value s (signed coefficients): true when some pair has s >= b2 (df 2) or
// s <= -b1 (df 1), with nb2 = -b2 and sb = b1 + b2 (both finite); two SNPs per
// packed instruction, as hit_fast_w.
template <int NS>
__device__ __forceinline__ bool hit_fast_w2(const uint32_t (&d0)[NS], const uint32_t (&d1)[NS],
                                            const ChunkMeta &m, int off, float nb2, float sb) {
  const uint64_t nt2 = pk2(__float_as_uint(nb2), __float_as_uint(nb2));
  const uint64_t sb2 = pk2(__float_as_uint(sb), __float_as_uint(sb));
  uint32_t hi = 0xffffffffu, lo = 0u;  // AND of the signs of s - b2, OR of those of s + b1
#pragma unroll
  for (int b = 0; b < NS / 16; ++b) {
    const uint64_t *al = reinterpret_cast<const uint64_t *>(m.alpha + off + 16 * b);
    const uint64_t *be = reinterpret_cast<const uint64_t *>(m.beta + off + 16 * b);
    const uint64_t *ga = reinterpret_cast<const uint64_t *>(m.gamma + off + 16 * b);
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
      const ulonglong2 A = *reinterpret_cast<const ulonglong2 *>(al + j);
      const ulonglong2 B = *reinterpret_cast<const ulonglong2 *>(be + j);
      const ulonglong2 G = *reinterpret_cast<const ulonglong2 *>(ga + j);
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int jj = 16 * b + 2 * (j + t);
        const uint64_t u2 = pk2(d0[jj], d0[jj + 1]);
        const uint64_t v2 = pk2(d1[jj], d1[jj + 1]);
        const uint64_t a2 = t ? A.y : A.x, b2 = t ? B.y : B.x, g2 = t ? G.y : G.x;
        const uint64_t w2 = ffma2(b2, v2, u2);
        const uint64_t e2 = fmul2(g2, v2);
        uint64_t q2 = ffma2(e2, v2, nt2);
        q2 = ffma2(fmul2(a2, w2), w2, q2);
        const uint64_t r2 = fadd2(q2, sb2);
        uint32_t qa, qb, ra, rb;
        upk2(q2, qa, qb);
        upk2(r2, ra, rb);
        hi &= qa & qb;
        lo |= ra | rb;
      }
    }
    if (b + 1 < NS / 16) asm volatile("" ::: "memory");
  }
  return (int)hi >= 0 || (int)lo < 0;
}

// Seed pass of a permutation batch in the plain form: the largest df-2 value and
// the most negative df-1 value of NS SNPs for this lane's trait, into smax / smin.
template <int NS>
__device__ __forceinline__ void range_w(const uint32_t (&d0)[NS], const uint32_t (&d1)[NS],
                                        const ChunkMeta &m, int off, float &smax, float &smin) {
#pragma unroll
  for (int b = 0; b < NS / 16; ++b) {
    const uint64_t *al = reinterpret_cast<const uint64_t *>(m.alpha + off + 16 * b);
    const uint64_t *be = reinterpret_cast<const uint64_t *>(m.beta + off + 16 * b);
    const uint64_t *ga = reinterpret_cast<const uint64_t *>(m.gamma + off + 16 * b);
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
      const ulonglong2 A = *reinterpret_cast<const ulonglong2 *>(al + j);
      const ulonglong2 B = *reinterpret_cast<const ulonglong2 *>(be + j);
      const ulonglong2 G = *reinterpret_cast<const ulonglong2 *>(ga + j);
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int jj = 16 * b + 2 * (j + t);
        const uint64_t u2 = pk2(d0[jj], d0[jj + 1]);
        const uint64_t v2 = pk2(d1[jj], d1[jj + 1]);
        const uint64_t a2 = t ? A.y : A.x, b2 = t ? B.y : B.x, g2 = t ? G.y : G.x;
        const uint64_t w2 = ffma2(b2, v2, u2);
        const uint64_t e2 = fmul2(g2, v2);
        const uint64_t s2 = ffma2(fmul2(a2, w2), w2, fmul2(e2, v2));
        uint32_t sa, sb;
        upk2(s2, sa, sb);
        smax = fmax3(smax, __uint_as_float(sa), __uint_as_float(sb));
        smin = fmin3(smin, __uint_as_float(sa), __uint_as_float(sb));
      }
    }
  }
}

// ---- hit events of the plain scan form, handled by the event warps ---------
// Several epilogue warps claim tickets at once, so one of them may claim an
// entry's use k while uses k-1, k-2 are still pending: a phase-parity wait
// cannot tell those apart.  A filler therefore waits on the entry's release count
// (uses the event warp has finished) reaching k; the uses of an entry are then
// filled in order, and its single consumer can wait on the full barrier by phase
// parity.
struct EvRing {
  EvEntry *ent;
  uint32_t bar0;                // ev_full[e] at bar0 + 8 e
  unsigned int *released;       // [kEvEntries] uses of each entry the event warps have finished
  unsigned long long *word;     // tickets claimed (low 40 bits), epilogue warps done (above)
  __device__ __forceinline__ uint32_t full(int e) const { return bar0 + 8u * (uint32_t)e; }
};
constexpr unsigned long long kEvTicketMask = (1ull << 40) - 1ull;

// Bounded wait of lane 0 until the entry of ticket t is free for its use t /
// kEvEntries; false on timeout or abort.
__device__ __forceinline__ bool ev_gate(const EvRing &ev, unsigned long long t, const ScanParams &p,
                                        uint32_t abort_addr) {
  const unsigned int k = (unsigned int)(t / kEvEntries);
  const volatile unsigned int *rel = ev.released + (t % kEvEntries);
  if (*rel >= k) return true;
  const long long t0 = clock64();
  while (*rel < k) {
    __nanosleep(128);
    int ab;
    asm volatile("ld.volatile.shared.u32 %0, [%1];" : "=r"(ab) : "r"(abort_addr) : "memory");
    if (ab) return false;
    if (clock64() - t0 > p.timeout_cycles) {
      asm volatile("st.volatile.shared.u32 [%0], %1;" ::"r"(abort_addr), "r"(1) : "memory");
      atomicOr(p.status, kDevTimeout);
      atomicMax(p.status + 1, 16u);
      return false;
    }
  }
  return true;
}

// An epilogue warp hands the traits of a half-block whose hot test found a
// candidate to the event warps: one entry per such trait lane (tickets claimed
// together), each with that lane's kEvSnps centred sums and constants and the
// SNPs' metadata (written by lanes 0..kEvSnps-1).  False if a wait gave up.
__device__ __forceinline__ bool ev_submit(const EvRing &ev, const uint32_t (&u)[kEvSnps],
                                          const uint32_t (&v)[kEvSnps], bool need,
                                          const ChunkMeta &m, int off, float tau, double cfac,
                                          int trait, int group, int ag, float b1, float b2,
                                          uint32_t id1, uint32_t id2, int nan, const ScanParams &p,
                                          uint32_t abort_addr, int lane) {
  uint32_t lanes = __ballot_sync(0xffffffffu, need);
  unsigned long long t = 0;
  if (lane == 0) t = atomicAdd(ev.word, (unsigned long long)__popc(lanes)) & kEvTicketMask;
  t = __shfl_sync(0xffffffffu, t, 0);
  // this lane's SNP metadata (lanes 0..kEvSnps-1), written into every entry
  const int jo = off + (lane & (kEvSnps - 1));
  const float al = m.alpha[jo], be = m.beta[jo], ga = m.gamma[jo];
  const int32_t sn = m.snp[jo];
  const uint32_t n01 = (uint32_t)m.n[0][jo] | ((uint32_t)m.n[1][jo] << 16);
  const uint32_t n2df = (uint32_t)m.n[2][jo] | ((uint32_t)m.df[jo] << 16);
  while (lanes) {
    const int L = __ffs((int)lanes) - 1;
    lanes &= lanes - 1u;
    int ok = 1;
    if (lane == 0) {
      ok = ev_gate(ev, t, p, abort_addr) ? 1 : 0;
      __threadfence_block();  // the event warp's reads of the old contents come first
    }
    if (!__shfl_sync(0xffffffffu, ok, 0)) return false;
    const int e = (int)(t % kEvEntries);
    EvEntry &E = ev.ent[e];
    if (lane < kEvSnps) {
      E.alpha[lane] = al;
      E.beta[lane] = be;
      E.gamma[lane] = ga;
      E.snp[lane] = sn;
      E.n01[lane] = n01;
      E.n2df[lane] = n2df;
    }
    if (lane == L) {
#pragma unroll
      for (int j = 0; j < kEvSnps; j += 4) {
        *reinterpret_cast<uint4 *>(E.u + j) = make_uint4(u[j], u[j + 1], u[j + 2], u[j + 3]);
        *reinterpret_cast<uint4 *>(E.v + j) = make_uint4(v[j], v[j + 1], v[j + 2], v[j + 3]);
      }
      E.cfac = cfac;
      E.tau = tau;
      E.trait = trait;
      E.group = group;
      E.ag = ag;
      E.b1 = b1;
      E.b2 = b2;
      E.id1 = id1;
      E.id2 = id2;
      E.nan = nan;
    }
    __threadfence_block();
    __syncwarp();
    if (lane == 0) mbar_arrive(ev.full(e));
    ++t;
  }
  return true;
}

// Group fields an event warp needs, cached across entries.
// Identity of a pair for exact-copy detection in permutation batches: a hash of
// its centred sums (copies of a SNP inside an LD block have the same sums and
// group sizes, hence the same statistic; pairs with equal sums and equal FP32
// form values but different group sizes would need an FP32 coincidence on top).
__device__ __forceinline__ uint32_t pair_id(int u, int v) {
  return (uint32_t)u * 0x9E3779B1u ^ (uint32_t)v * 0x85EBCA77u;
}

struct EvGroup {
  int index = -1;
  krux_hit *hits;
  HitAux *aux;
  unsigned long long *counter;
  int64_t capacity;
  uint16_t gid;
  double *minp_key;
  unsigned long long *minp_bound;
  int64_t rows;
  const uint16_t *nan_idx;  // NaN sample lists, N entries per trait
  const int8_t *geno;       // genotype rows (by output SNP index)
  int64_t ldg;
  int N;
};

__device__ __forceinline__ void ev_group(EvGroup &G, const ScanParams &p, int group) {
  if (group == G.index) return;
  const GroupDesc &g = p.groups[group];
  G.index = group;
  G.hits = g.hits;
  G.aux = g.aux;
  G.counter = g.counter;
  G.capacity = g.capacity;
  G.gid = (uint16_t)g.group_id;
  G.minp_key = g.minp_key;
  G.minp_bound = g.minp_bound;
  G.rows = g.rows_per_agroup;
  G.nan_idx = g.nan_idx;
  G.geno = g.geno;
  G.ldg = g.ldg;
  G.N = g.N;
}

// A permuted pair's entry (section "P-value calculation and empirical FDR
// correction": the minimum p of each permuted trait over all SNPs): lanes j <
// kEvSnps take the pairs past the submitting lane's bounds, decide them on their
// FP64 -ln p, raise the trait's key to the largest, and raise its class bounds
// (largest df-1 |s| and df-2 s of the pairs decided, less the margin: a later
// pair of the class below them cannot beat those pairs).  With the FDR histogram
// on, every pair at or above the band with p < P_c is counted in row ag.
__device__ __forceinline__ void ev_minp(const EvEntry &E, EvGroup &G, const ScanParams &p, int lane,
                                        float s, unsigned int &mcn, int ev_warp) {
  const int j = lane & (kEvSnps - 1);
  const bool valid = lane < kEvSnps && E.snp[j] >= 0;
  // E.b1, E.b2: the classes' largest decided values when the entry was filled,
  // E.id1, E.id2 the identities of the pairs that have them; exact copies of those
  // pairs are decided already
  const float keep = 1.f - p.margin;
  const float b1 = E.b1, b2 = E.b2;
  const uint32_t n01 = E.n01[j], n2df = E.n2df[j];
  const uint32_t pid = pair_id((int)E.u[j], (int)E.v[j]);
  bool cand = valid && ((s > b2 * keep && !(s == b2 && pid == E.id2)) ||
                        (-s > b1 * keep && !(-s == b1 && pid == E.id1)));
  // within a class the key grows with the value: only the entry's largest value
  // of each class, and values within the margin of it, can hold the class's best
  float c1 = cand && s < 0.f ? -s : 0.f, c2 = cand && s > 0.f ? s : 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    c1 = fmaxf(c1, __shfl_xor_sync(0xffffffffu, c1, o));
    c2 = fmaxf(c2, __shfl_xor_sync(0xffffffffu, c2, o));
  }
  cand = cand && (s > 0.f ? s >= c2 * keep : -s >= c1 * keep);
  const bool band = valid && p.fdr_hist != nullptr && fabsf(s) >= E.tau * (1.f - p.margin);
  const bool need = cand || band;
  const uint32_t bal = __ballot_sync(0xffffffffu, need);
  const unsigned int n = (unsigned int)__popc(bal);
  // identities of the pairs that hold the classes' largest values (the largest
  // identity among ties)
  const bool h1 = cand && s < 0.f && -s == c1, h2 = cand && s > 0.f && s == c2;
  const uint32_t w1 = __ballot_sync(0xffffffffu, h1), w2 = __ballot_sync(0xffffffffu, h2);
  const uint32_t i1 = __reduce_max_sync(0xffffffffu, h1 ? pid : 0u);
  const uint32_t i2 = __reduce_max_sync(0xffffffffu, h2 ? pid : 0u);
  if (mcn + n <= (unsigned int)p.mc_cap) {
    // the list has room: the FP64 work runs after the launch, in parallel
    if (need) {
      MinpPair r;
      r.u = (int32_t)E.u[j];
      r.v = (int32_t)E.v[j];
      r.n01 = n01;
      r.n2df = n2df;
      r.trait = E.trait;
      r.agb = E.ag | (band ? 1 << 16 : 0) | (cand ? 1 << 17 : 0);
      const size_t base = ((size_t)blockIdx.x * 2 + ev_warp) * (size_t)p.mc_cap;
      p.mc_list[base + mcn + (unsigned int)__popc(bal & ((1u << lane) - 1u))] = r;
    }
    mcn += n;
  } else {
    // full: decide here
    double key = -1.0;
    if (need) {
      const int df = (int)(n2df >> 16);
      if (df > 0 && E.cfac > 0.0)
        key = key64_of(kw_H64((int)E.u[j], (int)E.v[j], (int)(n01 & 0xffffu), (int)(n01 >> 16),
                              (int)(n2df & 0xffffu), E.cfac),
                       df);
    }
    if (band && key > -log(p.pthresh))
      atomicAdd(p.fdr_hist + (int64_t)E.ag * p.fdr_bins + fdr_bin(key, p.fdr_l0, p.fdr_w, p.fdr_bins),
                1ull);
    double kmax = cand ? key : -1.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) kmax = fmax(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
    if (lane == 0 && kmax > 0.0) {
      ev_group(G, p, E.group);
      atomicMax(reinterpret_cast<unsigned long long *>(G.minp_key + (int64_t)(E.ag - 1) * G.rows +
                                                       E.trait),
                (unsigned long long)__double_as_longlong(kmax));
    }
  }
  if (lane == 0) {
    ev_group(G, p, E.group);
    const int64_t idx = (int64_t)(E.ag - 1) * G.rows + E.trait;
    if (c1 > b1 && w1)
      atomicMax(G.minp_bound + 2 * idx, ((unsigned long long)__float_as_uint(c1) << 32) | i1);
    if (c2 > b2 && w2)
      atomicMax(G.minp_bound + 2 * idx + 1, ((unsigned long long)__float_as_uint(c2) << 32) | i2);
  }
}

// Event modes: the plain scan, a permutation batch, the plain scan with NaN.
enum EvMode { kEvPlain = 0, kEvPerm = 1, kEvNan = 2 };

// An event warp's work on one entry: lanes j < kEvSnps classify the pair (trait,
// SNP j) in the same FP32 form as the hot test (at or above the upper band edge:
// hit; inside the band: decided in FP64 from the exact sums) and the hits are
// appended in SNP order, one record per lane, into this warp's staging region of
// kEpiWarps / 2 segments of the CTA (`wn` records already there); what does not
// fit goes to the group's list through its counter.  For a trait with NaN
// samples (kEvNan) the pair's group sizes are first made exact (section "Handling
// missing values": N_i' counts the samples present for both): the genotypes of
// the trait's NaN samples at the SNP are taken off N_i, and the form is evaluated
// with those sizes and the df they leave.  Returns the number of hits.
template <int kMode>
__device__ __forceinline__ unsigned int ev_process(const EvEntry &E, EvGroup &G, const ScanParams &p,
                                                   unsigned int wn, int lane, int ev_warp,
                                                   unsigned int &mcn) {
  const int j = lane & (kEvSnps - 1);
  const bool act = lane < kEvSnps;
  const float tau = E.tau;
  const float u = E.u[j], v = E.v[j];
  const float w = fmaf(E.beta[j], v, u);
  const float sv = fmaf(E.alpha[j] * w, w, (E.gamma[j] * v) * v);
  float s = sv;
  uint32_t n01 = E.n01[j], n2df = E.n2df[j];
  if constexpr (kMode == kEvPerm) {
    if (E.ag > 0) {  // a permuted pair: min-p and FDR work, no hit record
      ev_minp(E, G, p, lane, sv, mcn, ev_warp);
      return 0u;
    }
    s = fabsf(sv);  // df-1 values are negated in permutation batches
  }
  if constexpr (kMode == kEvNan) {
    const int c = E.nan;
    if (c > 0) {
      ev_group(G, p, E.group);
      int n0 = (int)(n01 & 0xffffu), n1 = (int)(n01 >> 16), n2 = (int)(n2df & 0xffffu);
      const int sn = E.snp[j];
      if (act && sn >= 0) {
        const uint16_t *ni = G.nan_idx + (int64_t)E.trait * G.N;
        const int8_t *gr = G.geno + (int64_t)sn * G.ldg;
        for (int i = 0; i < c; i += 4) {  // four samples' loads in flight at once
          int k[4];
#pragma unroll
          for (int t = 0; t < 4; ++t) k[t] = i + t < c ? (int)ni[i + t] : -1;
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const int code = k[t] >= 0 ? (int)gr[k[t]] : -1;  // -1 (missing): in no group
            n0 -= code == 0;
            n1 -= code == 1;
            n2 -= code == 2;
          }
        }
      }
      const int df = df_of(n0, n1, n2);
      s = 0.f;
      if (act && sn >= 0 && df > 0) {
        const float w = -(u + v);
        float q = 0.f;
        if (n0 > 0) q += u * u / (float)n0;
        if (n1 > 0) q += v * v / (float)n1;
        if (n2 > 0) q += w * w / (float)n2;
        s = q / (df == 1 ? p.h1 : p.h2);
      }
      n01 = (uint32_t)n0 | ((uint32_t)n1 << 16);
      n2df = (uint32_t)n2 | ((uint32_t)df << 16);
    }
  }
  const bool cand = act && s + -tau * (1.f - p.margin) >= 0.f;
  bool hit = cand && s + -tau * (1.f + p.margin) >= 0.f;
  if (__any_sync(0xffffffffu, cand && !hit)) {  // inside the band: FP64 (rare)
    if (cand && !hit)
      hit = decide64_inl(u, v, (int)(n01 & 0xffffu), (int)(n01 >> 16), (int)(n2df & 0xffffu),
                         (int)(n2df >> 16), E.cfac, p.pthresh);
  }
  const uint32_t bal = __ballot_sync(0xffffffffu, hit);
  const unsigned int n = (unsigned int)__popc(bal);
  if (n == 0u) return 0u;
  ev_group(G, p, E.group);
  constexpr int kSegs = kEpiWarps / 2;  // staging segments per event warp
  const unsigned int cap = (unsigned int)(kSegs * p.seg_cap);
  const unsigned int over_from = wn > cap ? wn : cap;  // first index beyond the region
  const unsigned int n_over = wn + n > over_from ? wn + n - over_from : 0u;
  unsigned long long gbase = 0;
  if (lane == 0 && n_over > 0) gbase = atomicAdd(G.counter, (unsigned long long)n_over);
  gbase = __shfl_sync(0xffffffffu, gbase, 0);
  if (hit) {
    krux_hit rec;
    rec.trait = (uint32_t)E.trait;
    rec.snp = (uint32_t)E.snp[j];
    rec.d0 = (int32_t)u;
    rec.d1 = (int32_t)v;
    HitAux x;
    x.n0 = (uint16_t)(n01 & 0xffffu);
    x.n1 = (uint16_t)(n01 >> 16);
    x.n2 = (uint16_t)(n2df & 0xffffu);
    x.group = G.gid;
    const unsigned int idx = wn + (unsigned int)__popc(bal & ((1u << lane) - 1u));
    if (idx < cap) {
      const size_t seg0 = ((size_t)blockIdx.x * kEpiWarps + kSegs * ev_warp) * (size_t)p.seg_cap;
      st_hit(p.seg_hits + seg0 + idx, rec);
      st_aux(p.seg_aux + seg0 + idx, x);
    } else {
      const unsigned long long gi = gbase + (idx - over_from);
      if (gi < (unsigned long long)G.capacity) {
        st_hit(G.hits + gi, rec);
        st_aux(G.aux + gi, x);
      }
    }
  }
  return n;
}

// ---- markers with up to five groups ---------------------------------------
// Hot test of a warp's kEpiSnpsM SNPs of a 32-SNP chunk: true when some pair may
// lie at or above the lower band edge, Q/h_df = sum_i c_i D_i^2 + c_4 (sum_i D_i)^2
// >= tau (1 - margin), two SNPs per packed instruction.
__device__ __forceinline__ bool hit_fast_m(const uint32_t (&d)[kMaxCodeM][kEpiSnpsM],
                                           const ChunkMetaM &m, int h, float ntlo) {
  const int jb = kEpiSnpsM * h;
  const uint64_t nt2 = pk2(__float_as_uint(ntlo), __float_as_uint(ntlo));
  uint32_t acc = 0xffffffffu;
#pragma unroll
  for (int j = 0; j < kEpiSnpsM; j += 2) {
    uint64_t u[kMaxCodeM];
#pragma unroll
    for (int i = 0; i < kMaxCodeM; ++i) u[i] = pk2(d[i][j], d[i][j + 1]);
    const uint64_t s2 = fadd2(fadd2(u[0], u[1]), fadd2(u[2], u[3]));
    uint64_t q = nt2;
#pragma unroll
    for (int i = 0; i < kMaxCodeM; ++i) {
      const uint64_t c2 = *reinterpret_cast<const uint64_t *>(m.coef[i] + jb + j);
      q = ffma2(fmul2(c2, u[i]), u[i], q);
    }
    const uint64_t c4 = *reinterpret_cast<const uint64_t *>(m.coef[kMaxCodeM] + jb + j);
    q = ffma2(fmul2(c4, s2), s2, q);
    uint32_t qa, qb;
    upk2(q, qa, qb);
    acc &= qa & qb;
  }
  return (int)acc >= 0;
}

// FP64 decision for a pair inside the band: p < P_c from the exact sums.
__device__ __noinline__ bool decide64_m(const int *D, const ChunkMetaM &m, int jj, double cfac,
                                        double pthresh) {
  double Q = 0.0, S = 0.0;
  for (int i = 0; i < kMaxCodeM; ++i) {
    S += (double)D[i];
    if (m.n[i][jj] > 0) Q += (double)D[i] * (double)D[i] / (double)m.n[i][jj];
  }
  if (m.n[kMaxCodeM][jj] > 0) Q += S * S / (double)m.n[kMaxCodeM][jj];
  return chi2_tail64(cfac * Q, m.df[jj]) < pthresh;
}

// Rare path of a chunk of markers with up to five groups, called by the whole
// warp: classification of this lane's candidates and the warp's column-wise
// append into its staging segment (or the list), as hit_event does.  dv holds
// D_i of SNP j at dv[kEpiSnpsM * i + j] (i = 0..3).
__device__ __noinline__ unsigned int hit_event_m(const uint32_t *dv, bool mine, const ChunkMetaM &m,
                                                 int h, int trait, float ntlo, float nthi,
                                                 double cfac, const GroupDesc &g,
                                                 const ScanParams &p, unsigned int wn, int lane) {
  const int jb = kEpiSnpsM * h;
  uint32_t hm = 0;
  if (mine) {
    for (int j = 0; j < kEpiSnpsM; ++j) {
      const int jj = jb + j;
      if (m.snp[jj] < 0 || !in_cis_window(p, m.snp[jj], trait)) continue;
      float S = 0.f, q = 0.f;
      int D[kMaxCodeM];
      for (int i = 0; i < kMaxCodeM; ++i) {
        const float v = __uint_as_float(dv[kEpiSnpsM * i + j]);
        D[i] = (int)v;
        S += v;
        q = fmaf(m.coef[i][jj] * v, v, q);
      }
      q = fmaf(m.coef[kMaxCodeM][jj] * S, S, q);
      if (q + ntlo >= 0.f) {
        bool hit = q + nthi > 0.f;
        if (!hit) hit = decide64_m(D, m, jj, cfac, p.pthresh);
        if (hit) hm |= 1u << j;
      }
    }
  }
  const unsigned int total = __reduce_add_sync(0xffffffffu, (unsigned int)__popc(hm));
  if (total == 0u) return 0u;
  const unsigned int cap = (unsigned int)p.seg_cap;
  const unsigned int sbase = wn;
  const unsigned int over_from = sbase > cap ? sbase : cap;
  const unsigned int n_over = sbase + total > over_from ? sbase + total - over_from : 0u;
  unsigned long long gbase = 0;
  if (lane == 0 && n_over > 0) gbase = atomicAdd(g.counter, (unsigned long long)n_over);
  gbase = __shfl_sync(0xffffffffu, gbase, 0);
  const size_t seg0 = ((size_t)blockIdx.x * kEpiWarps + (threadIdx.x >> 5)) * cap;
  const uint32_t below_me = (1u << lane) - 1u;
  unsigned int run = sbase;
  uint32_t cols = __reduce_or_sync(0xffffffffu, hm);
  while (cols) {
    const int j = __ffs(cols) - 1;
    cols &= cols - 1u;
    const bool mine_j = (hm >> j) & 1u;
    const uint32_t bal = __ballot_sync(0xffffffffu, mine_j);
    if (mine_j) {
      const int jj = jb + j;
      const unsigned int idx = run + (unsigned int)__popc(bal & below_me);
      krux_hit r;
      r.trait = (uint32_t)trait;
      r.snp = (uint32_t)m.snp[jj];
      r.d0 = (int32_t)__uint_as_float(dv[j]);
      r.d1 = (int32_t)__uint_as_float(dv[kEpiSnpsM + j]);
      HitAux x;
      x.n0 = m.n[0][jj];
      x.n1 = m.n[1][jj];
      x.n2 = m.n[2][jj];
      x.group = (uint16_t)g.group_id;
      HitAux2 y;
      y.n3 = m.n[3][jj];
      y.n4 = m.n[4][jj];
      y.pad0_ = y.pad1_ = 0;
      y.d2 = (int32_t)__uint_as_float(dv[2 * kEpiSnpsM + j]);
      y.d3 = (int32_t)__uint_as_float(dv[3 * kEpiSnpsM + j]);
      if (idx < cap) {
        st_hit(p.seg_hits + seg0 + idx, r);
        st_aux(p.seg_aux + seg0 + idx, x);
        p.seg_aux2[seg0 + idx] = y;
      } else {
        const unsigned long long gi = gbase + (idx - over_from);
        if (gi < (unsigned long long)g.capacity) {
          st_hit(g.hits + gi, r);
          st_aux(g.aux + gi, x);
          g.aux2[gi] = y;
        }
      }
    }
    run += (unsigned int)__popc(bal);
  }
  return total;
}

// Hot filter bounds of one (permutation, trait): the running best -ln p turned
// into bounds on the form, |s| of df-1 SNPs and s of df-2 SNPs.
struct MinpState {
  float s1_lo, s2_lo;
};

// Bounds of the hot filter from the running best key: with key_lo = key (1 -
// margin), a df-2 SNP may beat it iff c2 s > key_lo, a df-1 SNP iff
// -ln erfc(sqrt(c1 |s| / 2)) > key_lo, i.e. c1 |s| > 2 erfcinv(exp(-key_lo))^2 (no
// transcendental left per chunk).  Past p ~ 1e-35 a lower bound of the inverse is
// used (the filter stays conservative).
__device__ __noinline__ MinpState minp_bounds(float key, float c1, float c2, float margin) {
  const float inf = __int_as_float(0x7f800000);
  const float klo = key * (1.f - margin);
  MinpState ms;
  ms.s2_lo = c2 > 0.f ? klo / c2 : inf;
  float h1 = 0.f;
  if (klo > 80.f) {
    h1 = 2.f * (klo - 0.5f * logf(3.14159265f * klo) - 1.f);
  } else if (klo > 0.f) {
    const float x = erfcinvf(expf(-klo));
    h1 = 2.f * x * x * (1.f - 1e-5f);
  }
  ms.s1_lo = c1 > 0.f ? h1 / c1 : inf;
  return ms;
}

// Largest df-2 form value (smax >= 0) and most negative df-1 form value
// (smin <= 0) of a permuted chunk half.
__device__ __forceinline__ void minp_range(const uint32_t (&d0)[kEpiSnps],
                                           const uint32_t (&d1)[kEpiSnps], const ChunkMeta &m,
                                           int h, float &smax_out, float &smin_out) {
  const uint64_t *al = reinterpret_cast<const uint64_t *>(m.alpha + kEpiSnps * h);
  const uint64_t *be = reinterpret_cast<const uint64_t *>(m.beta + kEpiSnps * h);
  const uint64_t *ga = reinterpret_cast<const uint64_t *>(m.gamma + kEpiSnps * h);
  float smax = 0.f, smin = 0.f;
#pragma unroll
  for (int j = 0; j < kEpiSnps / 2; j += 2) {
    const ulonglong2 A = *reinterpret_cast<const ulonglong2 *>(al + j);
    const ulonglong2 B = *reinterpret_cast<const ulonglong2 *>(be + j);
    const ulonglong2 G = *reinterpret_cast<const ulonglong2 *>(ga + j);
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int jj = 2 * (j + t);
      const uint64_t u2 = pk2(d0[jj], d0[jj + 1]);
      const uint64_t v2 = pk2(d1[jj], d1[jj + 1]);
      const uint64_t a2 = t ? A.y : A.x, b2 = t ? B.y : B.x, g2 = t ? G.y : G.x;
      const uint64_t w2 = ffma2(b2, v2, u2);
      const uint64_t e2 = fmul2(g2, v2);
      const uint64_t s2 = ffma2(fmul2(a2, w2), w2, fmul2(e2, v2));
      uint32_t sa, sb;
      upk2(s2, sa, sb);
      smax = fmax3(smax, __uint_as_float(sa), __uint_as_float(sb));
      smin = fmin3(smin, __uint_as_float(sa), __uint_as_float(sb));
    }
  }
  smax_out = smax;
  smin_out = smin;
}

// Seed bound of a step: FP32 -ln p of the largest values seen (ms holds them in
// seed mode), less twice the recheck margin so that it stays below the FP64 key of
// the pair that attains it.
__device__ __noinline__ double minp_seed_key(MinpState ms, float c1, float c2, float margin) {
  const float k = fmaxf(ms.s2_lo * c2, key1f(ms.s1_lo * c1));
  return (double)(k * (1.f - 2.f * margin));
}

// Class leader of one (permutation, trait) in a step: the pair with the largest
// form value among its df-1 SNPs (value |s|) or among its df-2 SNPs (value s).
// Within a class -ln p grows with the value (-ln p = c2 s for df 2, a function of
// c1 |s| that increases for df 1), so tracking the value needs no transcendental;
// the FP64 key is computed once, at the end of the step, or earlier on a near tie.
struct MinpCand {
  float s;        // FP32 value (0: no leader yet)
  float u, v;     // centred sums
  int n01;        // n0 | n1 << 16
  int n2df;       // n2 | df << 16
  double k64;     // FP64 -ln p once computed, else -1
};

// Leader state of one (permutation, trait) in a step.  Lives in local memory:
// touched only by the rare paths and at step boundaries.
struct MinpLead {
  MinpCand cls[2];  // [0]: df-1 SNPs, [1]: df-2 SNPs
  double exact;     // best FP64 key of the pairs decided exactly (traits with NaN), else -1
  double start;     // the global value at step start
  float c1, c2;     // H = c1 |s| for df-1 SNPs; -ln p = c2 s for df-2 SNPs
};

// FP64 -ln p of a pair from its exact sums (0 for degenerate pairs).
__device__ __noinline__ double lead_key64(float u, float v, int n0, int n1, int n2, int df,
                                          double cfac) {
  if (df <= 0 || !(cfac > 0.0)) return 0.0;
  return key64_of(kw_H64((int)u, (int)v, n0, n1, n2, cfac), df);
}

__device__ __forceinline__ double cand_key64(MinpCand &C, double cfac) {
  if (C.k64 < 0.0)
    C.k64 = lead_key64(C.u, C.v, C.n01 & 0xffff, C.n01 >> 16, C.n2df & 0xffff, C.n2df >> 16, cfac);
  return C.k64;
}

// Rare path of a permuted chunk half (trait without NaN): every SNP past the hot
// filter's bounds is offered to its class leader.  A clearly larger value (by more
// than the recheck margin) takes the lead without FP64; a near tie is decided on
// the FP64 keys.  The bound of the class then rises to the leader's value less the
// margin, so that only pairs that may beat the leader pass again.  With the FDR
// histogram on, every pair at or above the band gets its FP64 key and, if p < P_c,
// a count in row `row` of the histogram.
__device__ __noinline__ MinpState minp_event(const uint32_t *dv, const ChunkMeta &m, int h,
                                             double cfac, MinpLead *L, MinpState ms, float tau_lo,
                                             const ScanParams &p, int row) {
  const int jb = kEpiSnps * h;
  const float *al = m.alpha + jb, *be = m.beta + jb, *ga = m.gamma + jb;
  const float tie = p.margin;
  for (int j = 0; j < kEpiSnps; ++j) {
    if (m.snp[jb + j] < 0) continue;
    const float u = __uint_as_float(dv[j]), v = __uint_as_float(dv[kEpiSnps + j]);
    const float sv = kw_s(u, v, al[j], be[j], ga[j]);
    const bool lead = sv > ms.s2_lo || -sv > ms.s1_lo;
    const bool band = p.fdr_hist != nullptr && fabsf(sv) >= tau_lo;
    if (!lead && !band) continue;
    const int n0 = m.n[0][jb + j], n1 = m.n[1][jb + j], n2 = m.n[2][jb + j], df = m.df[jb + j];
    double key = -1.0;
    if (band) {
      key = lead_key64(u, v, n0, n1, n2, df, cfac);
      if (key > -log(p.pthresh))
        atomicAdd(p.fdr_hist + (int64_t)row * p.fdr_bins +
                      fdr_bin(key, p.fdr_l0, p.fdr_w, p.fdr_bins),
                  1ull);
    }
    if (!lead) continue;
    const int k = sv > 0.f ? 1 : 0;
    const float a = fabsf(sv);
    MinpCand &C = L->cls[k];
    bool take = a > C.s * (1.f + tie);
    // near tie with the leader: FP64, unless the pair repeats the leader's sums and
    // group sizes (copies of one SNP are common inside LD blocks) and so its key
    const bool same = u == C.u && v == C.v && (n0 | (n1 << 16)) == C.n01 &&
                      (n2 | (df << 16)) == C.n2df;
    if (!take && !same && a >= C.s * (1.f - tie)) {
      if (key < 0.0) key = lead_key64(u, v, n0, n1, n2, df, cfac);
      take = key > cand_key64(C, cfac);
    }
    if (take) {
      C.s = fmaxf(a, C.s);
      C.u = u;
      C.v = v;
      C.n01 = n0 | (n1 << 16);
      C.n2df = n2 | (df << 16);
      C.k64 = key;
    }
    if (k) ms.s2_lo = fmaxf(ms.s2_lo, C.s * (1.f - tie));
    else ms.s1_lo = fmaxf(ms.s1_lo, C.s * (1.f - tie));
  }
  return ms;
}

// Rare path of a permuted chunk half for a trait with NaN: the group sizes of each
// pair come from the genotype codes of its present samples, every pair is decided
// on its FP64 key (max into L->exact) and, with the FDR histogram on, counted.
__device__ __noinline__ void minp_event_nan(const uint32_t *dv, const ChunkMeta &m,
                                            const uint64_t *codes, int h, double cfac,
                                            int nan_cnt, const uint16_t *nan_idx, MinpLead *L,
                                            const ScanParams &p, int row) {
  const int jb = kEpiSnps * h;
  for (int j = 0; j < kEpiSnps; ++j) {
    if (m.snp[jb + j] < 0) continue;
    const float u = __uint_as_float(dv[j]), v = __uint_as_float(dv[kEpiSnps + j]);
    int n0, n1, n2;
    pair_counts(nan_cnt, nan_idx, m, codes, jb + j, n0, n1, n2);
    const double key = lead_key64(u, v, n0, n1, n2, df_of(n0, n1, n2), cfac);
    if (p.fdr_hist != nullptr && key > -log(p.pthresh))
      atomicAdd(p.fdr_hist + (int64_t)row * p.fdr_bins + fdr_bin(key, p.fdr_l0, p.fdr_w, p.fdr_bins),
                1ull);
    L->exact = fmax(L->exact, key);
  }
}

// End of a step: the best FP64 key of the step's leaders, if it beats the global
// value read at step start.
__device__ __noinline__ double minp_step_best(MinpLead *L, double cfac) {
  double best = L->exact;
  for (int k = 0; k < 2; ++k)
    if (L->cls[k].s > 0.f) best = fmax(best, cand_key64(L->cls[k], cfac));
  return best;
}

// Kernel forms: the plain scan, markers with up to five genotype groups (32-SNP
// chunks, ChunkMetaM), the permutation scan (groups with a min-p key), and the
// plain scan of rank sets with NaN (exact group sizes in the hot test); the
// producer and MMA warps are the same in all four.  Separate forms keep the
// state of one out of the registers of the others.
enum ScanForm {
  kFormScan = 0,
  kFormMulti = 1,
  kFormPerm = 2,
  kFormNan = 3,
  kFormScanPerm = 4,
  kFormScanNan = 5
};
// the plain scan form, its two-sided variant for permutation batches and its
// variant for expression with NaN
constexpr bool fast_form(int f) { return f == kFormScan || f == kFormScanPerm || f == kFormScanNan; }

// Warp roles of a kernel form: the epilogue warps first, then the producer and
// the MMA issuer (the plain scan form also has two idle warps after them).
template <int kForm>
struct ScanRoles {
  static constexpr int kEpi = fast_form(kForm) ? kFastEpiWarps : kEpiWarps;
  static constexpr int kProducer = kEpi;
  static constexpr int kMma = kEpi + 1;
  static constexpr int kThreads = fast_form(kForm) ? kFastThreads : kScanThreads;
};

template <int kForm>
__global__ void __launch_bounds__(ScanRoles<kForm>::kThreads, 1)
    krux_scan_kernel(const __grid_constant__ ScanParams p) {
  using R = ScanRoles<kForm>;
  extern __shared__ uint8_t smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t *sbase = smem_raw + (base - raw);
  const uint32_t a_tile_bytes = (uint32_t)p.a_tile_bytes;
  const uint32_t sA = base;
  const uint32_t sB = base + (uint32_t)p.nA * a_tile_bytes;
  ChunkMeta *smeta =
      reinterpret_cast<ChunkMeta *>(sbase + (size_t)p.nA * a_tile_bytes + (size_t)p.b_region);
  uint8_t *scodes = reinterpret_cast<uint8_t *>(smeta + p.nc);
  const uint32_t codes_stride = (uint32_t)p.kpad * 16u;
  uint8_t *stc = scodes + (size_t)p.nc * codes_stride;  // trait-constant ring
  // permutation form: per trait row, the min-p filter bounds of the current step
  // shared by the four warps that cover the row ((step tag << 32) | float bits;
  // df-1 bounds, then df-2 bounds)
  unsigned long long *sbound =
      reinterpret_cast<unsigned long long *>(stc + (size_t)kTcDepth * kTcBytes);
  uint64_t *bars = reinterpret_cast<uint64_t *>(sbound + 2 * kTileM);
  const uint32_t bar0 = smem_u32(bars);
  const int nA = p.nA, nc = p.nc;
  // barrier addresses
  auto a_full = [&](int s) { return bar0 + 8u * (uint32_t)s; };
  auto a_empty = [&](int s) { return bar0 + 8u * (uint32_t)(nA + s); };
  auto b_full = [&](int c) { return bar0 + 8u * (uint32_t)(2 * nA + c); };
  auto b_empty = [&](int c) { return bar0 + 8u * (uint32_t)(2 * nA + nc + c); };
  auto t_full = [&](int s) { return bar0 + 8u * (uint32_t)(2 * nA + 2 * nc + s); };
  auto t_empty = [&](int s) { return bar0 + 8u * (uint32_t)(2 * nA + 2 * nc + kTmemSlots + s); };
  const uint32_t drain = bar0 + 8u * (uint32_t)(2 * nA + 2 * nc + 2 * kTmemSlots);
  auto tc_full = [&](int e) { return bar0 + 8u * (uint32_t)(2 * nA + 2 * nc + 2 * kTmemSlots + 1 + e); };
  auto tc_empty = [&](int e) {
    return bar0 + 8u * (uint32_t)(2 * nA + 2 * nc + 2 * kTmemSlots + 1 + kTcDepth + e);
  };
  uint32_t *tmem_holder =
      reinterpret_cast<uint32_t *>(bars + 2 * nA + 2 * nc + 2 * kTmemSlots + 1 + 2 * kTcDepth);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_holder + 1);
  // plain scan form: the ring of hit-event buffers after everything else
  EvRing ev;
  {
    uint8_t *evr = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(tmem_holder) + 16u + 127u) & ~(uintptr_t)127u);
    ev.ent = reinterpret_cast<EvEntry *>(evr);
    ev.bar0 = smem_u32(evr + kEvEntries * sizeof(EvEntry));
    ev.released = reinterpret_cast<unsigned int *>(evr + kEvEntries * sizeof(EvEntry) + kEvEntries * 8);
    ev.word = reinterpret_cast<unsigned long long *>(evr + kEvEntries * sizeof(EvEntry) +
                                                     kEvEntries * 8 + kEvEntries * 4);
  }

  if (threadIdx.x == 0) {
    for (int s = 0; s < nA; ++s) {
      mbar_init(a_full(s), 1);
      mbar_init(a_empty(s), 1);
    }
    for (int c = 0; c < nc; ++c) {
      mbar_init(b_full(c), 1);
      mbar_init(b_empty(c), 1 + R::kEpi);
    }
    for (int s = 0; s < kTmemSlots; ++s) {
      mbar_init(t_full(s), 1);
      mbar_init(t_empty(s), R::kEpi);
    }
    mbar_init(drain, 1);
    for (int e = 0; e < kTcDepth; ++e) {
      mbar_init(tc_full(e), 1);
      mbar_init(tc_empty(e), R::kEpi);
    }
    *abort_flag = 0;
    if constexpr (fast_form(kForm)) {
      for (int e = 0; e < kEvEntries; ++e) {
        mbar_init(ev.full(e), 1);
        ev.released[e] = 0u;
      }
      *ev.word = 0ull;
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == R::kMma) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     smem_u32(tmem_holder))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  for (int i = threadIdx.x; i < 2 * kTileM; i += blockDim.x) sbound[i] = 0ull;
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_holder;
  const WaitCtl wc{abort_flag, p.status, p.timeout_cycles};
  // plain scan form: the registers of the producer warpgroup (warps 8-11) go to
  // the epilogue warps; each role's code sits under its own setmaxnreg

  if (warp == R::kProducer) {
    if constexpr (fast_form(kForm))
      asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kFastRegsLow) : "memory");
    if (lane == 0) {
      uint32_t a_stage = 0, a_phase = 0, b_bits = 0;
      uint32_t a_used = 0, a_last = 0, b_used = 0, b_last = 0;
      uint32_t tc_e = 0, tc_phase = 0, tc_used = 0, tc_last = 0;
      for (int it = blockIdx.x; it < p.n_items; it += gridDim.x) {
        const WorkItem w = p.items[it];
        const GroupDesc *g = p.groups + w.group;
        prefetch_map(&g->tmA);
        prefetch_map(&g->tmB);
        const int ncg = g->nc;
        const int nc_item = min(ncg, g->nchunks - w.btile * ncg);
        const uint32_t b_stride = (uint32_t)g->b_stride;
        const uint32_t abytes = atom_bytes(p.layout);
        const int ak = (int)atom_k(p.layout);
        const uint32_t b_tx = (uint32_t)g->n_atoms * abytes;
        const uint32_t codes_bytes = g->codes ? (uint32_t)g->codes_k * 16u : 0u;
        for (int c = 0; c < nc_item; ++c) {
          const uint32_t ph = (b_bits >> c) & 1u;
          if (!wait_bar(b_empty(c), ph ^ 1u, wc, 1)) goto producer_done;
          const int chunk = w.btile * ncg + c;
          mbar_expect_tx(b_full(c), b_tx + (uint32_t)sizeof(ChunkMeta) + codes_bytes);
          // paired groups interleave chunks 2j, 2j+1 per K atom: [atom][chunk of pair][128 rows]
          const uint32_t bbase = g->pair ? sB + (uint32_t)(c >> 1) * 2u * b_stride + (uint32_t)(c & 1) * abytes
                                         : sB + (uint32_t)c * b_stride;
          const uint32_t astep = g->pair ? 2u * abytes : abytes;
          for (int a = 0; a < g->n_atoms; ++a)
            tma_load_2d(bbase + (uint32_t)a * astep, &g->tmB, a * ak, g->b_row0 + chunk * kChunkRows,
                        b_full(c));
          bulk_load(smem_u32(smeta + c), g->meta + chunk, (uint32_t)sizeof(ChunkMeta), b_full(c));
          if (codes_bytes)
            bulk_load(smem_u32(scodes + (size_t)c * codes_stride), g->codes + (size_t)chunk * g->codes_k * 2,
                      codes_bytes, b_full(c));
          b_used |= 1u << c;
          b_last = (b_last & ~(1u << c)) | (ph << c);
          b_bits ^= 1u << c;
        }
        const int atoms_per_block = p.ka / ak;
        for (int step = w.step_begin; step < w.step_end; ++step) {
          const int ag = step / g->n_ttiles, tt = step - ag * g->n_ttiles;
          const int row0 = g->a_row0 + ag * g->rows_per_agroup + tt * kTileM;
          // the rank tile of this step, in K blocks of p.ka samples
          for (int kb = 0; kb < g->nkb; ++kb) {
            if (!wait_bar(a_empty(a_stage), a_phase ^ 1u, wc, 2)) goto producer_done;
            const int a0 = kb * atoms_per_block;
            const int na = min(atoms_per_block, g->n_atoms - a0);
            mbar_expect_tx(a_full(a_stage), (uint32_t)na * abytes);
            for (int a = 0; a < na; ++a)
              tma_load_2d(sA + (uint32_t)a_stage * a_tile_bytes + (uint32_t)a * abytes, &g->tmA,
                          (a0 + a) * ak, row0, a_full(a_stage));
            a_used |= 1u << a_stage;
            a_last = (a_last & ~(1u << a_stage)) | (a_phase << a_stage);
            if (++a_stage == (uint32_t)nA) {
              a_stage = 0;
              a_phase ^= 1u;
            }
          }
          // this step's per-trait constants into the ring (padded to whole tiles)
          if (!wait_bar(tc_empty(tc_e), tc_phase ^ 1u, wc, 8)) goto producer_done;
          {
            const bool with_key = g->minp_key != nullptr && ag > 0;
            constexpr uint32_t key_bytes = kForm == kFormScanPerm ? 2048u : 1024u;
            const uint32_t tx = 512u + 1024u + (g->nan_cnt ? 256u : 0u) + (with_key ? key_bytes : 0u);
            const uint32_t dst = smem_u32(stc + (size_t)tc_e * kTcBytes);
            const int64_t r0 = (int64_t)tt * kTileM;
            mbar_expect_tx(tc_full(tc_e), tx);
            bulk_load(dst, g->tau + r0, 512u, tc_full(tc_e));
            bulk_load(dst + 512u, g->cfac + r0, 1024u, tc_full(tc_e));
            if (with_key) {
              const int64_t kr = (int64_t)(ag - 1) * g->rows_per_agroup + r0;
              // the two-sided plain form reads the class bounds, the others the key
              if constexpr (kForm == kFormScanPerm)
                bulk_load(dst + 1536u, g->minp_bound + 2 * kr, 2048u, tc_full(tc_e));
              else
                bulk_load(dst + 1536u, g->minp_key + kr, 1024u, tc_full(tc_e));
            }
            if (g->nan_cnt) bulk_load(dst + 2560u, g->nan_cnt + r0, 256u, tc_full(tc_e));
            tc_used |= 1u << tc_e;
            tc_last = (tc_last & ~(1u << tc_e)) | (tc_phase << tc_e);
            if (++tc_e == (uint32_t)kTcDepth) {
              tc_e = 0;
              tc_phase ^= 1u;
            }
          }
        }
      }
    producer_done:
      // let every copy this thread issued land before the CTA can exit
      for (int s = 0; s < nA; ++s)
        if ((a_used >> s) & 1u) wait_drain(a_full(s), (a_last >> s) & 1u, p.status, 10);
      for (int c = 0; c < nc; ++c)
        if ((b_used >> c) & 1u) wait_drain(b_full(c), (b_last >> c) & 1u, p.status, 11);
      for (int e = 0; e < kTcDepth; ++e)
        if ((tc_used >> e) & 1u) wait_drain(tc_full(e), (tc_last >> e) & 1u, p.status, 13);
    }
    __syncwarp();
  } else if (warp == R::kMma && fast_form(kForm)) {
    // MMA issuer of the plain scan form: one N = 256 MMA chain per chunk pair (N =
    // 128 for an odd last chunk) into accumulator pair `ps` (TMEM columns ps *
    // 256 ..), released by the 8 epilogue warps as soon as they have loaded it
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kFastRegsLow) : "memory");
    if (lane == 0) {
      uint32_t a_stage = 0, a_phase = 0, b_bits = 0, ps = 0, ps_phase = 0;
      for (int it = blockIdx.x; it < p.n_items; it += gridDim.x) {
        const WorkItem w = p.items[it];
        const GroupDesc *g = p.groups + w.group;
        const int ncg = g->nc;
        const int nc_item = min(ncg, g->nchunks - w.btile * ncg);
        const uint32_t b_stride = (uint32_t)g->b_stride;
        const int ksteps = g->Np / 16;
        for (int step = w.step_begin; step < w.step_end; ++step) {
          if (!wait_bar(a_full(a_stage), a_phase, wc, 3)) goto fast_mma_done;
          tc_fence_after();
          const uint32_t a_tile = sA + a_stage * a_tile_bytes;
          for (int c = 0; c < nc_item; c += 2) {
            const bool two = c + 1 < nc_item;
            if (step == w.step_begin) {
              if (!wait_bar(b_full(c), (b_bits >> c) & 1u, wc, 4)) goto fast_mma_done;
              if (two && !wait_bar(b_full(c + 1), (b_bits >> (c + 1)) & 1u, wc, 4)) goto fast_mma_done;
            }
            if (!wait_bar(t_empty(ps), ps_phase ^ 1u, wc, 5)) goto fast_mma_done;
            tc_fence_after();
            // pair layout: [K atom][chunk of the pair][128 rows of 32 B]; a K step
            // moves the start address field only (it never carries)
            const uint32_t b_tile = sB + (uint32_t)(c >> 1) * 2u * b_stride;
            uint64_t da = umma_desc(a_tile, 1), db = umma_desc(b_tile, 1);
            const uint32_t d_tmem = tmem_base + ps * 256u;
            const uint32_t idesc = two ? kIdesc256 : kIdesc;
            tc_mma(d_tmem, da, db, idesc, 0u);
            for (int k = 1; k < ksteps; ++k) {
              da += 4096u >> 4;
              db += 8192u >> 4;
              tc_mma(d_tmem, da, db, idesc, 1u);
            }
            tc_commit(t_full(ps));
            ps ^= 1u;
            if (ps == 0u) ps_phase ^= 1u;
          }
          tc_commit(a_empty(a_stage));
          if (++a_stage == (uint32_t)nA) {
            a_stage = 0;
            a_phase ^= 1u;
          }
        }
        for (int c = 0; c < nc_item; ++c) {
          tc_commit(b_empty(c));
          b_bits ^= 1u << c;
        }
      }
    fast_mma_done:
      // all issued MMAs must finish before TMEM is released
      tc_commit(drain);
      wait_drain(drain, 0, p.status, 12);
    }
    __syncwarp();
  } else if (warp == R::kMma) {
    if (lane == 0) {
      uint32_t a_stage = 0, a_phase = 0, b_bits = 0, slot = 0, slot_phase = 0;
      for (int it = blockIdx.x; it < p.n_items; it += gridDim.x) {
        const WorkItem w = p.items[it];
        const GroupDesc *g = p.groups + w.group;
        const int ncg = g->nc;
        const int nc_item = min(ncg, g->nchunks - w.btile * ncg);
        const uint32_t b_stride = (uint32_t)g->b_stride;
        const int ksteps = g->Np / 16;
        const int kpb = p.ka / 16;  // K steps per block
        for (int step = w.step_begin; step < w.step_end; ++step) {
          if (g->pair && (slot & 1u)) {
            // paired accumulators start on an even slot: retire this one unused
            if (!wait_bar(t_empty(slot), slot_phase ^ 1u, wc, 14)) goto mma_done;
            tc_fence_after();
            tc_commit(t_full(slot));
            if (++slot == (uint32_t)kTmemSlots) {
              slot = 0;
              slot_phase ^= 1u;
            }
          }
          for (int kb = 0; kb < g->nkb; ++kb) {
            if (!wait_bar(a_full(a_stage), a_phase, wc, 3)) goto mma_done;
            tc_fence_after();
            const int k0 = kb * kpb;
            const int nk = min(kpb, ksteps - k0);
            const uint32_t a_tile = sA + a_stage * a_tile_bytes;
            for (int c = 0; c < nc_item;) {
              const bool two = g->pair && c + 1 < nc_item;
              uint32_t sc = slot + (uint32_t)c, ph = slot_phase;
              if (sc >= (uint32_t)kTmemSlots) {
                sc -= kTmemSlots;
                ph ^= 1u;
              }
              if (kb == 0) {
                for (int j = 0; j < (two ? 2 : 1); ++j) {
                  const uint32_t sj = sc + (uint32_t)j;  // sc is even when two: sj stays in range
                  if (step == w.step_begin) {
                    if (!wait_bar(b_full(c + j), (b_bits >> (c + j)) & 1u, wc, 4)) goto mma_done;
                  }
                  if (!wait_bar(t_empty(sj), ph ^ 1u, wc, 5)) goto mma_done;
                }
                tc_fence_after();
              }
              const uint32_t d_tmem = tmem_base + sc * 128u;
              // descriptors are built once per chunk and K block; a K step only moves
              // the start address field (bits 0-13, address >> 4), which never carries
              if (p.layout) {
                const uint32_t b_tile = g->pair ? sB + (uint32_t)(c >> 1) * 2u * b_stride
                                                : sB + (uint32_t)c * b_stride;
                const uint32_t bstep = g->pair ? 8192u : 4096u;
                const uint32_t idesc = two ? kIdesc256 : kIdesc;
                uint64_t da = umma_desc(a_tile, 1), db = umma_desc(b_tile + (uint32_t)k0 * bstep, 1);
                tc_mma(d_tmem, da, db, idesc, kb > 0 ? 1u : 0u);
                for (int k = 1; k < nk; ++k) {
                  da += 4096u >> 4;
                  db += bstep >> 4;
                  tc_mma(d_tmem, da, db, idesc, 1u);
                }
              } else {
                const uint32_t b_tile = sB + (uint32_t)c * b_stride;
                const uint64_t da = umma_desc(a_tile, 0), db = umma_desc(b_tile, 0);
                for (int k = 0; k < nk; ++k) {
                  const uint64_t oa = (uint64_t)(kstep_off(0, k) >> 4);
                  const uint64_t ob = (uint64_t)(kstep_off(0, k0 + k) >> 4);
                  tc_mma(d_tmem, da + oa, db + ob, kIdesc, (kb > 0 || k > 0) ? 1u : 0u);
                }
              }
              if (kb == g->nkb - 1) {
                tc_commit(t_full(sc));
                if (two) tc_commit(t_full(sc + 1u));
              }
              c += two ? 2 : 1;
            }
            tc_commit(a_empty(a_stage));
            if (++a_stage == (uint32_t)nA) {
              a_stage = 0;
              a_phase ^= 1u;
            }
          }
          slot += (uint32_t)nc_item;
          if (slot >= (uint32_t)kTmemSlots) {
            slot -= kTmemSlots;
            slot_phase ^= 1u;
          }
        }
        for (int c = 0; c < nc_item; ++c) {
          tc_commit(b_empty(c));
          b_bits ^= 1u << c;
        }
      }
    mma_done:
      // all issued MMAs must finish before TMEM is released
      tc_commit(drain);
      wait_drain(drain, 0, p.status, 12);
    }
    __syncwarp();
  } else if constexpr (fast_form(kForm)) {
    // epilogue warps of the plain scan form: warp 4k + q owns lane quarter q of
    // kFastSnps SNPs of one chunk of every accumulator pair; it loads their D_0 and
    // D_1 with one wait, releases the pair at once, then runs the hot test (and,
    // when a lane has a candidate, the hit event) on the registers
    if (warp >= R::kEpi) {  // the two event warps of the producer warpgroup
      asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kFastRegsLow) : "memory");
      const int e = warp - (R::kMma + 1);
      unsigned int wn = 0;  // hits this event warp has appended to its staging region
      unsigned int mcn = 0;  // permuted pairs it has passed on to the deferred FP64 pass
      EvGroup G;
      for (unsigned long long t = (unsigned long long)e;; t += 2) {
        const int b = (int)(t % kEvEntries);
        const uint32_t ph = (uint32_t)((t / kEvEntries) & 1ull);
        // lane 0 waits until ticket t is filled or no more tickets can come
        int got = 0;
        if (lane == 0) {
          const long long t0 = clock64();
          while (true) {
            if (mbar_try_wait_sleep(ev.full(b), ph, 20000u)) {
              got = 1;
              break;
            }
            if (*abort_flag) break;
            const unsigned long long wv = *reinterpret_cast<volatile unsigned long long *>(ev.word);
            if ((wv >> 40) >= (unsigned long long)kFastEpiWarps && t >= (wv & kEvTicketMask)) break;
            if (clock64() - t0 > p.timeout_cycles) {
              *abort_flag = 1;
              atomicOr(p.status, kDevTimeout);
              atomicMax(p.status + 1, 17u);
              break;
            }
          }
        }
        got = __shfl_sync(0xffffffffu, got, 0);
        if (!got) break;
        wn += ev_process<kForm == kFormScanPerm ? kEvPerm : (kForm == kFormScanNan ? kEvNan : kEvPlain)>(
            ev.ent[b], G, p, wn, lane, e, mcn);
        __syncwarp();
        if (lane == 0) {  // this use of the buffer is finished
          __threadfence_block();
          atomicAdd(ev.released + b, 1u);
        }
      }
      if constexpr (kForm == kFormScanPerm)
        if (lane == 0 && p.mc_cnt != nullptr) p.mc_cnt[blockIdx.x * 2 + e] = min(mcn, (unsigned int)p.mc_cap);
      if (lane == 0 && p.seg_cap > 0) {  // this event warp's staging segments
        constexpr int kSegs = kEpiWarps / 2;
        const unsigned int cap = (unsigned int)p.seg_cap;
        for (int sgi = 0; sgi < kSegs; ++sgi) {
          const unsigned int lo = cap * (unsigned int)sgi;
          p.seg_cnt[blockIdx.x * kEpiWarps + kSegs * e + sgi] = wn > lo ? min(wn - lo, cap) : 0u;
        }
      }
    } else {
      asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kFastRegsHigh) : "memory");
      constexpr int kPerChunk = kChunkSnps / kFastSnps;  // warps per chunk and lane quarter
      const int q = warp & 3, k = warp >> 2;
      const int h = k / kPerChunk;                     // chunk of the pair
      const int off = kFastSnps * (k % kPerChunk);     // first SNP within the chunk
      const int row = 32 * q + lane;
      const uint32_t abort_addr = smem_u32(const_cast<const int *>(abort_flag));
      const uint32_t lane_cols =
          tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(128 * h + off);
      uint32_t ps = 0, ps_phase = 0, b_bits = 0, tc_e = 0, tc_phase = 0;
      constexpr int kH = kFastSnps / 2;
      // permutation batches (two-sided form): per class (df 1: -s, df 2: s) the
      // largest value decided so far for this lane's trait in the current step and
      // the identity of the pair that has it; a pair may pass when its value exceeds
      // the decided one less the margin (at most `cap`: the band's lower edge while
      // FDR counts are on).  The unpermuted group tests both signs against tau.
      constexpr bool kTwo = kForm == kFormScanPerm;
      constexpr bool kNan = kForm == kFormScanNan;
      constexpr float kBoundMin = 1e-30f, kBoundMax = 1e30f;
      // expression with NaN: the bound of this lane's trait is coefficient set
      // nset - 1 of the chunk's block (0: the chunk metadata's exact coefficients;
      // -1: more NaN samples than any set covers, every pair goes to the exact
      // test).  The warp first tests all its lanes with the loosest set any of them
      // needs (wset: one address for the whole warp), and only when some lane
      // passes, and the lanes' sets differ (mixed), each lane again with its own set
      // (lanes reading different addresses cost several shared-memory passes per
      // load).  One register: nset + 1 in bits 0-3, wset in bits 4-7, mixed bit 8,
      // the trait's NaN count from bit 9.
      int nsw = 1;
      int cpair = 0;  // the chunk pair_slot works on, within the work item
      float mx1 = 0.f, mx2 = 0.f, bnd1 = 0.f, bnd2 = 0.f;  // decided values, hot-test bounds
      uint32_t id1 = 0u, id2 = 0u;
      int ag = 0;  // the step's rank-matrix group (> 0: a permutation)
      // seed pass: this lane's largest df-2 value and df-1 |value| in the step and
      // the 16-SNP blocks (positions in the group's SNP order) that hold them
      const bool seed = kTwo && p.seed_bound != 0;
      float smax = 0.f, smin = 0.f;
      int pos2 = 0, pos1 = 0;
      int chunk0 = 0;  // the work item's first chunk in the group
      // the hot test's bounds from the decided values (cap: the band's lower edge
      // while FDR counts are on, else none)
      auto set_bounds = [&](float cap) {
        const float keep = 1.f - p.margin;
        bnd1 = fminf(fminf(mx1 * keep, cap), kBoundMax);
        bnd2 = fminf(fminf(mx2 * keep, cap), kBoundMax);
      };
      auto test = [&](const uint32_t(&x0)[kH], const uint32_t(&x1)[kH], const ChunkMeta &mc, int o,
                      float ntlo) -> bool {
        if constexpr (kTwo) {
          return hit_fast_w2<kH>(x0, x1, mc, o, -bnd2, bnd1 + bnd2);
        } else if constexpr (kNan) {
          const uint8_t *blk = scodes + (size_t)cpair * codes_stride;
          const int wset = (nsw >> 4) & 15, nset = (nsw & 15) - 1;
          const float *cw = wset > 0 ? coef_set(blk, wset - 1)->alpha : mc.alpha;
          bool need = hit_fast_wc<kH>(x0, x1, cw, cw + kChunkSnps, cw + 2 * kChunkSnps, o, ntlo);
          if (((nsw >> 8) & 1) && __any_sync(0xffffffffu, need)) {
            const float *cf = nset > 0 ? coef_set(blk, nset - 1)->alpha : mc.alpha;
            need = hit_fast_wc<kH>(x0, x1, cf, cf + kChunkSnps, cf + 2 * kChunkSnps, o, ntlo) && need;
          }
          return need;
        } else {
          return hit_fast_w<kH>(x0, x1, mc, o, ntlo);
        }
      };
      // a permuted block past the hot test: the lane's pairs that still need the
      // event warps (past the bounds but not exact copies of a class's decided pair
      // -- copies are common inside LD blocks -- or in the FDR band), and the
      // classes' new largest values with the identities of their pairs
      auto minp_filter = [&](const uint32_t(&x0)[kH], const uint32_t(&x1)[kH], const ChunkMeta &mc,
                             int o, float tau, float &n1, float &n2, uint32_t &k1,
                             uint32_t &k2) -> bool {
        const float tlo = p.fdr_hist != nullptr ? tau * (1.f - p.margin) : kBoundMax;
        const float b1 = bnd1, b2 = bnd2;
        bool any = false;
        n1 = mx1;
        n2 = mx2;
        k1 = id1;
        k2 = id2;
        for (int j = 0; j < kH; ++j) {
          const float u = __uint_as_float(x0[j]), v = __uint_as_float(x1[j]);
          const float sv = kw_s(u, v, mc.alpha[o + j], mc.beta[o + j], mc.gamma[o + j]);
          bool c2 = sv > b2, c1 = -sv > b1;
          uint32_t pid = 0u;
          if (c1 || c2) pid = pair_id((int)u, (int)v);
          c2 = c2 && !(sv == mx2 && pid == id2);
          c1 = c1 && !(-sv == mx1 && pid == id1);
          any = any || c1 || c2 || fabsf(sv) >= tlo;
          if (c2 && sv > n2) {
            n2 = sv;
            k2 = pid;
          }
          if (c1 && -sv > n1) {
            n1 = -sv;
            k1 = pid;
          }
        }
        return any;
      };
      // one accumulator pair: wait for it, load this warp's two halves (the second
      // while the first is tested), release it, test the second half, hand any
      // candidate half-block to the event warps; false if a wait gave up
      auto pair_slot = [&](uint32_t ps, uint32_t phase, const ChunkMeta &mc, float tau,
                           double cfac, float ntlo, int trait, int group) -> bool {
        if (!__all_sync(0xffffffffu, wait_bar_p(t_full(ps), phase, p, abort_addr, 7))) return false;
        tc_fence_after();
        uint32_t a0[kH], a1[kH], b0[kH], b1[kH];
        const uint32_t taddr = lane_cols + ps * 256u;
        tmem_ld_half(taddr, a0, a1);
        tmem_wait_ld();
        tmem_ld_half(taddr + (uint32_t)kH, b0, b1);
        if constexpr (kTwo) {
          if (seed) {
            const int pos = (chunk0 + cpair) * kChunkSnps + off;
            float hi = 0.f, lo = 0.f;
            range_w<kH>(a0, a1, mc, off, hi, lo);
            tmem_wait_ld();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(t_empty(ps));
            if (hi > smax) { smax = hi; pos2 = pos; }
            if (lo < smin) { smin = lo; pos1 = pos; }
            hi = 0.f;
            lo = 0.f;
            range_w<kH>(b0, b1, mc, off + kH, hi, lo);
            if (hi > smax) { smax = hi; pos2 = pos + kH; }
            if (lo < smin) { smin = lo; pos1 = pos + kH; }
            return true;
          }
        }
        const bool need_a = test(a0, a1, mc, off, ntlo);
        tmem_wait_ld();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(t_empty(ps));
        const bool need_b = test(b0, b1, mc, off + kH, ntlo);
        if (__any_sync(0xffffffffu, need_a)) {
          bool real = need_a;
          float n1 = 0.f, n2 = 0.f;
          uint32_t k1 = 0u, k2 = 0u;
          if constexpr (kTwo)
            if (ag > 0 && need_a) real = minp_filter(a0, a1, mc, off, tau, n1, n2, k1, k2);
          if (__any_sync(0xffffffffu, real) &&
              !ev_submit(ev, a0, a1, real, mc, off, tau, cfac, trait, group, ag, mx1, mx2, id1, id2,
                         kNan ? nsw >> 9 : 0, p, abort_addr, lane))
            return false;
          if constexpr (kTwo)
            if (ag > 0 && real) {
              mx1 = n1;
              mx2 = n2;
              id1 = k1;
              id2 = k2;
              set_bounds(p.fdr_hist != nullptr ? tau * (1.f - p.margin) : kBoundMax);
            }
        }
        if (__any_sync(0xffffffffu, need_b)) {
          bool real = need_b;
          float n1 = 0.f, n2 = 0.f;
          uint32_t k1 = 0u, k2 = 0u;
          if constexpr (kTwo)
            if (ag > 0 && need_b) real = minp_filter(b0, b1, mc, off + kH, tau, n1, n2, k1, k2);
          if (__any_sync(0xffffffffu, real) &&
              !ev_submit(ev, b0, b1, real, mc, off + kH, tau, cfac, trait, group, ag, mx1, mx2, id1, id2,
                         kNan ? nsw >> 9 : 0, p, abort_addr, lane))
            return false;
          if constexpr (kTwo)
            if (ag > 0 && real) {
              mx1 = n1;
              mx2 = n2;
              id1 = k1;
              id2 = k2;
              set_bounds(p.fdr_hist != nullptr ? tau * (1.f - p.margin) : kBoundMax);
            }
        }
        return true;
      };
      for (int it = blockIdx.x; it < p.n_items; it += gridDim.x) {
        const WorkItem w = p.items[it];
        const GroupDesc &g = p.groups[w.group];
        const int g_nc = g.nc, g_ntt = g.n_ttiles;
        const int nc_item = min(g_nc, g.nchunks - w.btile * g_nc);
        // this warp's chunks of the B tile (h and 2 + h) must have landed
        {
          bool ok = true;
          for (int c = h; c < nc_item; c += 2) ok = ok && wait_bar_p(b_full(c), (b_bits >> c) & 1u, p, abort_addr, 6);
          if (!__all_sync(0xffffffffu, ok)) goto epi_done_scan;
        }
        int tt = w.step_begin % g_ntt;  // trait tile of the step
        chunk0 = w.btile * g_nc;
        for (int step = w.step_begin; step < w.step_end; ++step) {
          // this step's trait constants, staged by the producer (copied out at once)
          if (!__all_sync(0xffffffffu, wait_bar_p(tc_full(tc_e), tc_phase, p, abort_addr, 9)))
            goto epi_done_scan;
          const uint8_t *tcp = stc + (size_t)tc_e * kTcBytes;
          const float tau = reinterpret_cast<const float *>(tcp)[row];
          const double cfac = reinterpret_cast<const double *>(tcp + 512)[row];
          const int trait = tt * kTileM + row;
          if constexpr (kNan) {
            const int nan_c = g.nan_cnt ? (int)reinterpret_cast<const uint16_t *>(tcp + 2560)[row] : 0;
            const int nset = nan_c == 0 ? 0 : (nan_c <= kNanCMax ? nan_set_of(nan_c) + 1 : -1);
            const int wset = (int)__reduce_max_sync(0xffffffffu, (unsigned)max(nset, 0));
            const bool mixed = __any_sync(0xffffffffu, nset >= 0 && nset != wset);
            nsw = (nset + 1) | (wset << 4) | (mixed ? 256 : 0) | (nan_c << 9);
          }
          if constexpr (kTwo) {
            // unpermuted group: both signs against tau (less the margin); a
            // permuted one: the classes' decided values staged for the step
            ag = step / g_ntt;
            if (ag > 0) {
              // per class: (value bits << 32) | identity, as little-endian words
              const uint4 bb = reinterpret_cast<const uint4 *>(tcp + 1536)[row];
              mx1 = fmaxf(__uint_as_float(bb.y), kBoundMin);
              id1 = bb.x;
              mx2 = fmaxf(__uint_as_float(bb.w), kBoundMin);
              id2 = bb.z;
              set_bounds(p.fdr_hist != nullptr ? tau * (1.f - p.margin) : kBoundMax);
            } else {
              mx1 = tau;
              mx2 = tau;
              id1 = 0u;
              id2 = 0u;
              set_bounds(kBoundMax);
            }
            smax = 0.f;
            smin = 0.f;
            pos2 = 0;
            pos1 = 0;
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(tc_empty(tc_e));
          if (++tc_e == (uint32_t)kTcDepth) {
            tc_e = 0;
            tc_phase ^= 1u;
          }
          float ntlo = -tau * (1.f - p.margin);
          // (a trait beyond the last set: +inf lets every pair through)
          if constexpr (kNan)
            if ((nsw & 15) == 0 && tau < kBoundMax) ntlo = __int_as_float(0x7f800000);
          {
            for (int c0 = 0; c0 < nc_item; c0 += 2) {
              const int c = c0 + h;
              if (c < nc_item) {
                cpair = c;
                if (!pair_slot(ps, ps_phase, smeta[c], tau, cfac, ntlo, trait, w.group))
                  goto epi_done_scan;
              } else {  // an odd last chunk leaves warps 8-15 idle: release only
                if (!__all_sync(0xffffffffu, wait_bar_p(t_full(ps), ps_phase, p, abort_addr, 7)))
                  goto epi_done_scan;
                tc_fence_after();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(t_empty(ps));
              }
              ps ^= 1u;
              if (ps == 0u) ps_phase ^= 1u;
            }
          }
          if constexpr (kTwo) {
            // seed pass: the step's largest values and their blocks (the largest
            // over all steps is decided exactly after the launch)
            if (seed && ag > 0 && trait < g.T) {
              unsigned long long *rp =
                  g.minp_seed + 2 * ((int64_t)(ag - 1) * g.rows_per_agroup + trait);
              if (smin < 0.f)
                atomicMax(rp, ((unsigned long long)__float_as_uint(-smin) << 32) | (uint32_t)(pos1 + 1));
              if (smax > 0.f)
                atomicMax(rp + 1, ((unsigned long long)__float_as_uint(smax) << 32) | (uint32_t)(pos2 + 1));
            }
          }
          if (++tt == g_ntt) tt = 0;
        }
        // the chunks' metadata is no longer needed
        __syncwarp();
        if (lane == 0)
          for (int c = 0; c < nc_item; ++c) mbar_arrive(b_empty(c));
        for (int c = 0; c < nc_item; ++c) b_bits ^= 1u << c;
      }
    epi_done_scan:
      tc_fence_before();
      __syncwarp();
      if (lane == 0) atomicAdd(ev.word, 1ull << 40);  // no more events from this warp
    }
  } else {
    // epilogue warps
    const int q = warp & 3, h = warp >> 2;  // lane quarter, SNP group of the chunk
    uint32_t slot = 0, slot_phase = 0, b_bits = 0, tc_e = 0, tc_phase = 0;
    unsigned int wn = 0;  // hits this warp has appended to its staging segment
    uint32_t step_tag = 0;  // steps begun by this warp (the same count in every epilogue warp)
    for (int it = blockIdx.x; it < p.n_items; it += gridDim.x) {
      const WorkItem w = p.items[it];
      const GroupDesc &g = p.groups[w.group];
      const int nc_item = min(g.nc, g.nchunks - w.btile * g.nc);
      const int g_ntt = g.n_ttiles, g_T = g.T, g_N = g.N;
      const bool g_has_nan = g.nan_cnt != nullptr;
      for (int step = w.step_begin; step < w.step_end; ++step) {
        const int ag = step / g_ntt, tt = step - ag * g_ntt;
        if (g.pair && (slot & 1u)) {
          // the MMA warp retired this slot unused (paired accumulators start even)
          if (!__all_sync(0xffffffffu, wait_bar(t_full(slot), slot_phase, wc, 15))) goto epi_done;
          __syncwarp();
          if (lane == 0) mbar_arrive(t_empty(slot));
          if (++slot == (uint32_t)kTmemSlots) {
            slot = 0;
            slot_phase ^= 1u;
          }
        }
        if constexpr (kForm == kFormPerm) ++step_tag;
        // this step's trait constants, staged by the producer
        if (!__all_sync(0xffffffffu, wait_bar(tc_full(tc_e), tc_phase, wc, 9))) goto epi_done;
        const uint8_t *tcp = stc + (size_t)tc_e * kTcBytes;
        const int row = 32 * q + lane;
        EpiTrait et;
        et.trait = tt * kTileM + row;
        et.valid = et.trait < g_T;
        const float tau = reinterpret_cast<const float *>(tcp)[row];
        et.ntlo = -tau * (1.f - p.margin);
        et.nthi = -tau * (1.f + p.margin);
        et.cfac = reinterpret_cast<const double *>(tcp + 512)[row];
        et.nan_cnt = g_has_nan ? (int)reinterpret_cast<const uint16_t *>(tcp + 2560)[row] : 0;
        et.nan_idx = g_has_nan && et.valid
                         ? g.nan_idx + ag * g.nan_ag_stride + (int64_t)et.trait * g_N
                         : nullptr;
        const bool minp_mode = kForm == kFormPerm && g.minp_key != nullptr && ag > 0;
        const bool seed_pass = kForm == kFormPerm && p.seed_bound != 0;
        // traits with NaN (form kFormNan): the hot test's bounds on sum_i D_i^2 / n_i'
        float nan_q1 = 0.f, nan_q2 = 0.f;
        if (kForm == kFormNan) {
          const float cf = (float)et.cfac;
          nan_q1 = cf > 0.f ? p.h1 * (1.f - p.margin) / cf : __int_as_float(0x7f800000);
          nan_q2 = cf > 0.f ? p.h2 * (1.f - p.margin) / cf : __int_as_float(0x7f800000);
        }
        // with the FDR histogram on, permuted pairs at or above the band are counted
        const float fdr_tau_lo = p.fdr_hist != nullptr ? -et.ntlo : __int_as_float(0x7f800000);
        // min-p state: FP64 work only in permuted groups (FP64 issue is slow here)
        MinpState ms;
        MinpLead lead;
        double *key_ptr = nullptr;
        if (minp_mode) {
          lead.start = 0.0;
          lead.c1 = 0.f;
          lead.c2 = 0.f;
          if (et.valid) {
            lead.c1 = (float)et.cfac * p.h1;  // FP32: these only scale the filter
            lead.c2 = (float)et.cfac * p.h2 * 0.5f;
            key_ptr = g.minp_key + (int64_t)(ag - 1) * g.rows_per_agroup + et.trait;
            lead.start = reinterpret_cast<const double *>(tcp + 1536)[row];
          }
          for (int k = 0; k < 2; ++k) {
            lead.cls[k].s = 0.f;
            lead.cls[k].u = __int_as_float(0x7fc00000);  // NaN: equal to no pair
            lead.cls[k].k64 = -1.0;
          }
          lead.exact = -1.0;
          ms = minp_bounds((float)lead.start, lead.c1, lead.c2, p.margin);
          if (seed_pass) {  // ms tracks the largest values instead
            ms.s1_lo = 0.f;
            ms.s2_lo = 0.f;
          }
        }
        for (int c = 0; c < nc_item; ++c) {
          bool ok = true;
          if (step == w.step_begin) ok = wait_bar(b_full(c), (b_bits >> c) & 1u, wc, 6);
          ok = ok && wait_bar(t_full(slot), slot_phase, wc, 7);
          if (!__all_sync(0xffffffffu, ok)) goto epi_done;
          tc_fence_after();
          if constexpr (kForm == kFormMulti) {
            // markers with up to five groups: this warp's 8 SNPs of a 32-SNP chunk,
            // D_i of SNP j in column 32 i + j (i = 0..3)
            uint32_t dd[kMaxCodeM][kEpiSnpsM];
            const uint32_t tb =
                tmem_base + ((uint32_t)(32 * q) << 16) + slot * 128u + (uint32_t)(kEpiSnpsM * h);
#pragma unroll
            for (int i = 0; i < kMaxCodeM; ++i) tmem_ld8(tb + (uint32_t)(kChunkSnpsM * i), dd[i]);
            tmem_wait_ld();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(t_empty(slot));
            if (++slot == (uint32_t)kTmemSlots) {
              slot = 0;
              slot_phase ^= 1u;
            }
            const ChunkMetaM &mm = *reinterpret_cast<const ChunkMetaM *>(&smeta[c]);
            const bool need = hit_fast_m(dd, mm, h, et.ntlo);
            if (__any_sync(0xffffffffu, need)) {
              uint32_t dv[kMaxCodeM * kEpiSnpsM];
#pragma unroll
              for (int i = 0; i < kMaxCodeM; ++i)
#pragma unroll
                for (int j = 0; j < kEpiSnpsM; ++j) dv[kEpiSnpsM * i + j] = dd[i][j];
              wn += hit_event_m(dv, need && et.valid, mm, h, et.trait, et.ntlo, et.nthi, et.cfac,
                                g, p, wn, lane);
            }
          } else {
            uint32_t d0[kEpiSnps], d1[kEpiSnps];
            const uint32_t taddr =
                tmem_base + ((uint32_t)(32 * q) << 16) + slot * 128u + (uint32_t)(kEpiSnps * h);
            tmem_ld16(taddr, d0);
            tmem_ld16(taddr + 64u, d1);
            tmem_wait_ld();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(t_empty(slot));
            if (++slot == (uint32_t)kTmemSlots) {
              slot = 0;
              slot_phase ^= 1u;
            }
            const uint64_t *codes =
                g.codes ? reinterpret_cast<const uint64_t *>(scodes + (size_t)c * codes_stride) : nullptr;
            const ChunkMeta &mc = smeta[c];
            bool need;
            if (minp_mode && seed_pass) {
              // seed pass: only the range of the values (traits with NaN sit out)
              float smax, smin;
              minp_range(d0, d1, mc, h, smax, smin);
              ms.s2_lo = fmaxf(ms.s2_lo, smax);
              ms.s1_lo = fmaxf(ms.s1_lo, -smin);
              need = false;
            } else if (minp_mode) {
              if (!et.valid) {
                need = false;
              } else if (et.nan_cnt > 0) {
                need = true;
              } else {
                float smax, smin;
                minp_range(d0, d1, mc, h, smax, smin);
                need = smax > ms.s2_lo || -smin > ms.s1_lo || fmaxf(smax, -smin) >= fdr_tau_lo;
                if (need) {
                  // the row's bounds from the other warps' leaders of this step first
                  const unsigned long long b1 = sbound[row], b2 = sbound[kTileM + row];
                  if ((uint32_t)(b1 >> 32) == step_tag)
                    ms.s1_lo = fmaxf(ms.s1_lo, __uint_as_float((uint32_t)b1));
                  if ((uint32_t)(b2 >> 32) == step_tag)
                    ms.s2_lo = fmaxf(ms.s2_lo, __uint_as_float((uint32_t)b2));
                  need = smax > ms.s2_lo || -smin > ms.s1_lo || fmaxf(smax, -smin) >= fdr_tau_lo;
                }
              }
            }
            else if (kForm == kFormNan && et.nan_cnt > 0)
              need = p.dense || hit_fast_nan(d0, d1, mc, h, codes, et.nan_cnt, et.nan_idx,
                                             nan_q1, nan_q2);
            else
              need = p.dense || et.nan_cnt > 0 ||
                     (p.signed_coef ? hit_fast<true>(d0, d1, mc, h, et.ntlo)
                                    : hit_fast<false>(d0, d1, mc, h, et.ntlo));
            if (__any_sync(0xffffffffu, need)) {
              // rare paths work on a local copy of the accumulators
              uint32_t dv[2 * kEpiSnps];
  #pragma unroll
              for (int j = 0; j < kEpiSnps; ++j) {
                dv[j] = d0[j];
                dv[kEpiSnps + j] = d1[j];
              }
              if (minp_mode) {
                if (need) {
                  if (et.nan_cnt > 0)
                    minp_event_nan(dv, mc, codes, h, et.cfac, et.nan_cnt, et.nan_idx, &lead, p, ag);
                  else {
                    ms = minp_event(dv, mc, h, et.cfac, &lead, ms, fdr_tau_lo, p, ag);
                    const unsigned long long tag = (unsigned long long)step_tag << 32;
                    atomicMax(&sbound[row], tag | __float_as_uint(ms.s1_lo));
                    atomicMax(&sbound[kTileM + row], tag | __float_as_uint(ms.s2_lo));
                  }
                }
              } else if (__any_sync(0xffffffffu, p.dense || et.nan_cnt > 0)) {
                hit_slow(dv, need, mc, codes, h, et.trait, et.valid, et.ntlo, et.nthi, et.cfac,
                         et.nan_cnt, et.nan_idx, g, p, lane);
              } else {
                if constexpr (kForm == kFormPerm)
                  wn += hit_event_cols(dv, need && et.valid, mc, h, et.trait, et.ntlo, et.nthi,
                                       et.cfac, g, p, wn, lane);
                else
                  wn += hit_event(dv, need && et.valid, mc, h, et.trait, et.ntlo, et.nthi, et.cfac,
                                  g, p, wn, lane);
              }
            }
          }
          if (step == w.step_end - 1) {
            __syncwarp();
            if (lane == 0) mbar_arrive(b_empty(c));
          }
        }
        if (minp_mode && key_ptr != nullptr) {
          const double k64 = !seed_pass         ? minp_step_best(&lead, et.cfac)
                             : et.nan_cnt == 0 ? minp_seed_key(ms, lead.c1, lead.c2, p.margin)
                                               : -1.0;
          if (k64 > lead.start)
            atomicMax(reinterpret_cast<unsigned long long *>(key_ptr),
                      (unsigned long long)__double_as_longlong(k64));
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(tc_empty(tc_e));
        if (++tc_e == (uint32_t)kTcDepth) {
          tc_e = 0;
          tc_phase ^= 1u;
        }
      }
      for (int c = 0; c < nc_item; ++c) b_bits ^= 1u << c;
    }
  epi_done:
    tc_fence_before();
    if (lane == 0 && p.seg_cap > 0)
      p.seg_cnt[blockIdx.x * kEpiWarps + warp] = min(wn, (unsigned int)p.seg_cap);
  }

  __syncthreads();
  if (warp == R::kMma) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem_base) : "memory");
  }
}

// Appends every staging segment (one per epilogue warp of every CTA) after the
// directly appended hits: block b copies segment b to offset
// direct + sum_{c<b} seg_cnt[c] (entries past the capacity are dropped); block 0
// also writes the exact total.
__global__ void seg_compact_kernel(const krux_hit *__restrict__ seg_hits,
                                   const HitAux *__restrict__ seg_aux,
                                   const HitAux2 *__restrict__ seg_aux2,
                                   const unsigned int *__restrict__ seg_cnt, int n_seg,
                                   int seg_cap, const unsigned long long *__restrict__ direct,
                                   krux_hit *__restrict__ out, HitAux *__restrict__ out_aux,
                                   HitAux2 *__restrict__ out_aux2, int64_t capacity,
                                   unsigned long long *total) {
  __shared__ unsigned long long part[2][8];
  const int b = blockIdx.x;
  unsigned long long before = 0, all = 0;
  for (int c = threadIdx.x; c < n_seg; c += blockDim.x) {
    const unsigned long long v = seg_cnt[c];
    all += v;
    if (c < b) before += v;
  }
  for (int o = 16; o > 0; o >>= 1) {
    before += __shfl_xor_sync(0xffffffffu, before, o);
    all += __shfl_xor_sync(0xffffffffu, all, o);
  }
  if ((threadIdx.x & 31) == 0) {
    part[0][threadIdx.x >> 5] = before;
    part[1][threadIdx.x >> 5] = all;
  }
  __syncthreads();
  unsigned long long off = *direct, tot = *direct;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
    off += part[0][w];
    tot += part[1][w];
  }
  if (b == 0 && threadIdx.x == 0) *total = tot;
  const unsigned int n = seg_cnt[b];
  const size_t s0 = (size_t)b * seg_cap;
  for (unsigned int i = threadIdx.x; i < n; i += blockDim.x) {
    const unsigned long long o = off + i;
    if (o < (unsigned long long)capacity) {
      st_hit(out + o, ld_hit(seg_hits + s0 + i));
      st_aux(out_aux + o, ld_aux(seg_aux + s0 + i));
      if (out_aux2 != nullptr) out_aux2[o] = seg_aux2[s0 + i];
    }
  }
}

// 1/n in FP64 for n = 0..kMaxN (entry 0 unused): the finalisation multiplies
// instead of dividing (FP64 division is slow on this part).
__device__ double c_rcp[kMaxN + 1];  // (global, read through L1: the indices differ by lane)

// FP64 statistic and p-value of each stored hit, from its exact centred sums.
__device__ __forceinline__ void finalize_one(const krux_hit *__restrict__ hits,
                                             const HitAux *__restrict__ aux,
                                             const HitAux2 *__restrict__ aux2, int64_t i,
                                             const double *const *__restrict__ cfac_by_group,
                                             double *__restrict__ H, double *__restrict__ P,
                                             unsigned long long *fdr_hist, int fdr_bins,
                                             double fdr_l0, double fdr_w, double pthresh) {
  const krux_hit r = ld_hit(hits + i);
  const HitAux a = ld_aux(aux + i);
  const double cf = cfac_by_group[a.group][r.trait];
  int df;
  double Q;
  if (aux2 == nullptr) {
    df = df_of(a.n0, a.n1, a.n2);
    const double D0 = (double)r.d0, D1 = (double)r.d1, D2 = -(double)(r.d0 + r.d1);
    Q = D0 * D0 * __ldg(&c_rcp[a.n0]);
    Q = fma(D1 * D1, __ldg(&c_rcp[a.n1]), Q);
    Q = fma(D2 * D2, __ldg(&c_rcp[a.n2]), Q);
  } else {  // five groups: D_4 = -(D_0 + D_1 + D_2 + D_3)
    const HitAux2 b = aux2[i];
    const int n[5] = {a.n0, a.n1, a.n2, b.n3, b.n4};
    const double D[5] = {(double)r.d0, (double)r.d1, (double)b.d2, (double)b.d3,
                         -((double)r.d0 + (double)r.d1 + (double)b.d2 + (double)b.d3)};
    int groups = 0;
    Q = 0.0;
    for (int k = 0; k < 5; ++k) {
      groups += n[k] > 0;
      Q = fma(D[k] * D[k], __ldg(&c_rcp[n[k]]), Q);
    }
    df = groups > 0 ? groups - 1 : 0;
  }
  const double h = cf * Q;
  H[i] = h;
  double pv;
  if (df < 1 || df > 2) {  // markers with more groups: df 3, 4
    pv = chi2_tail64(h, df);
  } else {
    pv = kw_p_report(h, df);
    if (pv >= pthresh) pv = kw_p64(h, df);  // a hit's p stays below P_c as decided
  }
  P[i] = pv;
  if (fdr_hist != nullptr)  // row 0: the real data's hits by -log10 p bin
    atomicAdd(fdr_hist + fdr_bin(key64_of(h, df), fdr_l0, fdr_w, fdr_bins), 1ull);
}

__global__ void finalize_kernel(const krux_hit *__restrict__ hits, const HitAux *__restrict__ aux,
                                int64_t n, const double *const *__restrict__ cfac_by_group,
                                double *__restrict__ H, double *__restrict__ P,
                                unsigned long long *fdr_hist, int fdr_bins, double fdr_l0,
                                double fdr_w, double pthresh) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    finalize_one(hits, aux, nullptr, i, cfac_by_group, H, P, fdr_hist, fdr_bins, fdr_l0, fdr_w,
                 pthresh);
}

// The same over min(*count, capacity) hits, the count read on the device (no host
// round trip between the scan and the finalisation; capturable in a graph).
__global__ void finalize_dev_kernel(const krux_hit *__restrict__ hits,
                                    const HitAux *__restrict__ aux,
                                    const HitAux2 *__restrict__ aux2,
                                    const unsigned long long *__restrict__ count, int64_t capacity,
                                    const double *const *__restrict__ cfac_by_group,
                                    double *__restrict__ H, double *__restrict__ P,
                                    unsigned long long *fdr_hist, int fdr_bins, double fdr_l0,
                                    double fdr_w, double pthresh) {
  const unsigned long long c = *count;
  const int64_t n = c < (unsigned long long)capacity ? (int64_t)c : capacity;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    finalize_one(hits, aux, aux2, i, cfac_by_group, H, P, fdr_hist, fdr_bins, fdr_l0, fdr_w, pthresh);
}

// The deferred FP64 pass of a plain-form permutation launch: every listed pair's
// -ln p (section "P-value calculation and empirical FDR correction"), the largest
// per (permutation, trait) into the key, and pairs of the FDR band with p < P_c
// into the histogram row of their permutation.
__global__ void minp_cands_kernel(const MinpPair *__restrict__ list, const unsigned int *__restrict__ cnt,
                                  int n_lists, int cap, const double *__restrict__ cfac, int rows_pad,
                                  double lp, double *key, unsigned long long *fdr_hist, int fdr_bins,
                                  double fdr_l0, double fdr_w) {
  for (int l = blockIdx.y; l < n_lists; l += gridDim.y) {
    const unsigned int n = min(cnt[l], (unsigned int)cap);
    for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
      const MinpPair r = list[(size_t)l * cap + i];
      const int df = (int)(r.n2df >> 16), ag = r.agb & 0xffff;
      const double cf = cfac[r.trait];
      if (df <= 0 || !(cf > 0.0)) continue;
      const double k = key64_of(kw_H64(r.u, r.v, (int)(r.n01 & 0xffffu), (int)(r.n01 >> 16),
                                       (int)(r.n2df & 0xffffu), cf),
                                df);
      if (r.agb & (1 << 17))
        atomicMax(reinterpret_cast<unsigned long long *>(key + (int64_t)(ag - 1) * rows_pad + r.trait),
                  (unsigned long long)__double_as_longlong(k));
      if ((r.agb & (1 << 16)) && fdr_hist != nullptr && k > lp)
        atomicAdd(fdr_hist + (int64_t)ag * fdr_bins + fdr_bin(k, fdr_l0, fdr_w, fdr_bins), 1ull);
    }
  }
}

// After a plain-form seed pass of a permutation batch: one warp per (permutation
// q, trait, class) whose seed record names a 16-SNP block.  The block's centred
// rank sums are recomputed as integers (the permuted centred ranks against the
// genotype indicators, as the contraction forms them), its largest value of the
// class is found again with the fast test's FP32 expression, that pair's FP64 -ln p
// (section "P-value calculation and empirical FDR correction") is folded into the
// key, and its value becomes the class's largest decided value.
__global__ void seed_decide_kernel(const unsigned long long *__restrict__ rec,
                                   const __half *__restrict__ stack, int rows_pad, int Np, int N,
                                   int T, int P, const int8_t *__restrict__ geno, int64_t ldg,
                                   int64_t snp_begin, int64_t n_snps,
                                   const ChunkMeta *__restrict__ meta,
                                   const double *__restrict__ cfac, double *key,
                                   unsigned long long *bound) {
  const int lane = threadIdx.x & 31;
  const int64_t nrec = (int64_t)P * T * 2;
  for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < nrec;
       r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int cls = (int)(r & 1);
    const int64_t qt = r >> 1;
    const int q = (int)(qt / T), trait = (int)(qt % T);
    const int64_t idx = (int64_t)q * rows_pad + trait;
    const unsigned long long v = rec[2 * idx + cls];
    if (v == 0ull) continue;
    const int64_t pos0 = (int64_t)(uint32_t)(v & 0xffffffffull) - 1;
    const __half *a = stack + ((int64_t)(1 + q) * rows_pad + trait) * Np;
    float best = 0.f;
    int bj = -1, bu = 0, bv = 0;
    for (int j = 0; j < 16 && pos0 + j < n_snps; ++j) {
      const int64_t pos = pos0 + j;
      const int8_t *g = geno + (snp_begin + pos) * ldg;
      int d0 = 0, d1 = 0;
      for (int k = lane; k < N; k += 32) {
        const int ak = (int)__half2float(a[k]);
        const int8_t gk = g[k];
        d0 += gk == 0 ? ak : 0;
        d1 += gk == 1 ? ak : 0;
      }
      d0 = __reduce_add_sync(0xffffffffu, d0);
      d1 = __reduce_add_sync(0xffffffffu, d1);
      const ChunkMeta &m = meta[pos / kChunkSnps];
      const int w = (int)(pos % kChunkSnps);
      if (m.snp[w] < 0) continue;
      const float sv = kw_s((float)d0, (float)d1, m.alpha[w], m.beta[w], m.gamma[w]);
      const float val = cls ? sv : -sv;
      if (val > best) {
        best = val;
        bj = j;
        bu = d0;
        bv = d1;
      }
    }
    if (lane == 0 && bj >= 0) {
      const int64_t pos = pos0 + bj;
      const ChunkMeta &m = meta[pos / kChunkSnps];
      const int w = (int)(pos % kChunkSnps);
      const int df = m.df[w];
      const double cf = cfac[trait];
      if (df > 0 && cf > 0.0) {
        const double k64 = key64_of(kw_H64(bu, bv, m.n[0][w], m.n[1][w], m.n[2][w], cf), df);
        atomicMax(reinterpret_cast<unsigned long long *>(key + idx),
                  (unsigned long long)__double_as_longlong(k64));
      }
      const uint32_t pid = pair_id(bu, bv);
      atomicMax(bound + 2 * idx + cls, ((unsigned long long)__float_as_uint(best) << 32) | pid);
    }
  }
}

// minimum p of each (permutation, trait) from its best -ln p (key rows of ld entries)
__global__ void minp_from_key_kernel(const double *__restrict__ key, double *__restrict__ minp,
                                     int P, int T, int ld) {
  const int64_t n = (int64_t)P * T;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    minp[i] = exp(-key[(i / T) * ld + i % T]);
}

}  // namespace

cudaError_t launch_seg_compact(const krux_hit *seg_hits, const HitAux *seg_aux,
                               const HitAux2 *seg_aux2, const unsigned int *seg_cnt, int n_seg,
                               int seg_cap, const unsigned long long *direct, krux_hit *out,
                               HitAux *out_aux, HitAux2 *out_aux2, int64_t capacity,
                               unsigned long long *total, cudaStream_t s) {
  if (n_seg <= 0) return cudaSuccess;
  seg_compact_kernel<<<n_seg, 256, 0, s>>>(seg_hits, seg_aux, seg_aux2, seg_cnt, n_seg, seg_cap,
                                           direct, out, out_aux, out_aux2, capacity, total);
  return cudaGetLastError();
}

cudaError_t launch_minp_from_key(const double *key, double *minp, int P, int T, int ld,
                                 cudaStream_t s) {
  const int64_t n = (int64_t)P * T;
  if (n <= 0) return cudaSuccess;
  int grid = (int)((n + 255) / 256);
  if (grid > 4096) grid = 4096;
  minp_from_key_kernel<<<grid, 256, 0, s>>>(key, minp, P, T, ld);
  return cudaGetLastError();
}

cudaError_t launch_minp_cands(const MinpPair *list, const unsigned int *cnt, int n_lists, int cap,
                              const double *cfac, int rows_pad, double pthresh, double *key,
                              unsigned long long *fdr_hist, int fdr_bins, double fdr_l0,
                              double fdr_w, cudaStream_t s) {
  if (n_lists <= 0 || cap <= 0) return cudaSuccess;
  const dim3 grid((unsigned)((cap + 255) / 256 < 64 ? (cap + 255) / 256 : 64),
                  (unsigned)(n_lists < 65535 ? n_lists : 65535));
  minp_cands_kernel<<<grid, 256, 0, s>>>(list, cnt, n_lists, cap, cfac, rows_pad, -log(pthresh), key,
                                         fdr_hist, fdr_bins, fdr_l0, fdr_w);
  return cudaGetLastError();
}

cudaError_t launch_seed_decide(const unsigned long long *rec, const __half *stack, int rows_pad,
                               int Np, int N, int T, int P, const int8_t *geno, int64_t ldg,
                               int64_t snp_begin, int64_t n_snps, const ChunkMeta *meta,
                               const double *cfac, double *key, unsigned long long *bound,
                               cudaStream_t s) {
  const int64_t warps = (int64_t)P * T * 2;
  if (warps <= 0) return cudaSuccess;
  const int64_t blocks = (warps + 7) / 8;
  const int grid = (int)(blocks < 65535 ? blocks : 65535);
  seed_decide_kernel<<<grid, 256, 0, s>>>(rec, stack, rows_pad, Np, N, T, P, geno, ldg, snp_begin,
                                          n_snps, meta, cfac, key, bound);
  return cudaGetLastError();
}

size_t scan_smem_bytes(int nc, int nA, int kpad) {
  return scan_smem_bytes2(nc, nA, (size_t)128 * kpad * 2, (size_t)nc * 128 * kpad * 2, kpad);
}

size_t scan_smem_bytes2(int nc, int nA, size_t a_tile_bytes, size_t b_region, int codes_k) {
  return 1024 + (size_t)nA * a_tile_bytes + b_region + (size_t)nc * sizeof(ChunkMeta) +
         (size_t)nc * codes_k * 16 + (size_t)kTcDepth * kTcBytes + 16 * (size_t)kTileM +
         8 * (size_t)(2 * nA + 2 * nc + 2 * kTmemSlots + 1 + 2 * kTcDepth) + 16;
}

bool fast_form_ok();
cudaError_t scan_set_smem_all(size_t smem);

cudaError_t scan_set_smem(size_t smem) {
  (void)fast_form_ok();  // its one-time check happens here, before any graph capture
  // the attribute is per device: skip the calls when it already has this value
  static std::atomic<size_t> last[64];
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64 &&
      last[dev].load(std::memory_order_acquire) == smem + 1)
    return cudaSuccess;
  cudaError_t e = scan_set_smem_all(smem);
  if (e == cudaSuccess && dev >= 0 && dev < 64) last[dev].store(smem + 1, std::memory_order_release);
  return e;
}

cudaError_t scan_set_smem_all(size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(krux_scan_kernel<kFormScan>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(krux_scan_kernel<kFormScanNan>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(krux_scan_kernel<kFormScanPerm>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(krux_scan_kernel<kFormMulti>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(krux_scan_kernel<kFormNan>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(krux_scan_kernel<kFormPerm>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// The kernel form launch_scan_only picks for these parameters (the ScanForm value).
int scan_form_of(const ScanParams &p) {
  if (p.multi) return kFormMulti;
  if (p.perm) return p.fast && fast_form_ok() ? kFormScanPerm : kFormPerm;
  if (p.fast && fast_form_ok()) return p.fast_nan ? kFormScanNan : kFormScan;
  return kFormNan;
}

cudaError_t launch_scan_only(const ScanParams &p, int grid, size_t smem, cudaStream_t s) {
  if (p.multi)
    krux_scan_kernel<kFormMulti><<<grid, kScanThreads, smem, s>>>(p);
  else if (p.perm && p.fast && fast_form_ok())
    krux_scan_kernel<kFormScanPerm><<<grid, kFastThreads, smem, s>>>(p);
  else if (p.perm)
    krux_scan_kernel<kFormPerm><<<grid, kScanThreads, smem, s>>>(p);
  else if (p.fast && p.fast_nan && fast_form_ok())
    krux_scan_kernel<kFormScanNan><<<grid, kFastThreads, smem, s>>>(p);
  else if (p.fast && fast_form_ok())
    krux_scan_kernel<kFormScan><<<grid, kFastThreads, smem, s>>>(p);
  else
    // the general form: traits with NaN, dense output, cis window, provisional
    // hits, unpaired chunks
    krux_scan_kernel<kFormNan><<<grid, kScanThreads, smem, s>>>(p);
  return cudaGetLastError();
}

// The plain scan form moves registers between its warpgroups with setmaxnreg,
// which is sound only if the kernel was built with exactly the launch register
// count the split assumes (else an increase could wait for registers that were
// never there): checked once, before its first launch.
bool fast_form_ok() {
  static std::atomic<int> ok{-1};
  int v = ok.load(std::memory_order_acquire);
  if (v < 0) {
    // the plain-form kernels were built at the register count their warp roles'
    // setmaxnreg split assumes
    cudaFuncAttributes a, b, c;
    v = cudaFuncGetAttributes(&a, krux_scan_kernel<kFormScan>) == cudaSuccess &&
                cudaFuncGetAttributes(&b, krux_scan_kernel<kFormScanPerm>) == cudaSuccess &&
                cudaFuncGetAttributes(&c, krux_scan_kernel<kFormScanNan>) == cudaSuccess &&
                a.numRegs == kFastRegsLaunch && a.maxThreadsPerBlock >= kFastThreads &&
                b.numRegs == kFastRegsLaunch && b.maxThreadsPerBlock >= kFastThreads &&
                c.numRegs == kFastRegsLaunch && c.maxThreadsPerBlock >= kFastThreads
            ? 1
            : 0;
    ok.store(v, std::memory_order_release);
  }
  return v == 1;
}

cudaError_t launch_scan(const ScanParams &p, int grid, size_t smem, cudaStream_t s) {
  cudaError_t e = scan_set_smem(smem);
  if (e != cudaSuccess) return e;
  return launch_scan_only(p, grid, smem, s);
}

cudaError_t finalize_prepare() {
  // bit d: the table is on device d (callers on several host threads may race
  // to upload it; the upload is idempotent, the mask update atomic)
  static std::atomic<unsigned long long> uploaded{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 64 && ((uploaded.load(std::memory_order_acquire) >> dev) & 1ull)) return cudaSuccess;
  double t[kMaxN + 1];
  t[0] = 0.0;  // empty groups have D_i = 0 and contribute nothing
  for (int k = 1; k <= kMaxN; ++k) t[k] = 1.0 / (double)k;
  e = cudaMemcpyToSymbol(c_rcp, t, sizeof t);
  if (e != cudaSuccess) return e;
  if (dev < 64) uploaded.fetch_or(1ull << dev, std::memory_order_acq_rel);
  return cudaSuccess;
}

cudaError_t launch_finalize(const krux_hit *hits, const HitAux *aux, int64_t n,
                            const double *const *cfac_by_group, double *H, double *p,
                            cudaStream_t s, unsigned long long *fdr_hist, int fdr_bins,
                            double fdr_l0, double fdr_w, double pthresh) {
  if (n <= 0) return cudaSuccess;
  cudaError_t e = finalize_prepare();
  if (e != cudaSuccess) return e;
  int grid = (int)((n + 255) / 256);
  if (grid > 152 * 8) grid = 152 * 8;
  finalize_kernel<<<grid, 256, 0, s>>>(hits, aux, n, cfac_by_group, H, p, fdr_hist, fdr_bins, fdr_l0,
                                       fdr_w, pthresh);
  return cudaGetLastError();
}

cudaError_t launch_finalize_dev(const krux_hit *hits, const HitAux *aux, const HitAux2 *aux2,
                                const unsigned long long *count, int64_t capacity,
                                const double *const *cfac_by_group, double *H, double *p,
                                int sm_count, cudaStream_t s, unsigned long long *fdr_hist,
                                int fdr_bins, double fdr_l0, double fdr_w, double pthresh) {
  if (capacity <= 0) return cudaSuccess;
  int grid = sm_count * 4;
  const int64_t need = (capacity + 255) / 256;
  if (need < grid) grid = (int)need;
  finalize_dev_kernel<<<grid, 256, 0, s>>>(hits, aux, aux2, count, capacity, cfac_by_group, H, p,
                                           fdr_hist, fdr_bins, fdr_l0, fdr_w, pthresh);
  return cudaGetLastError();
}

}  // namespace krux

