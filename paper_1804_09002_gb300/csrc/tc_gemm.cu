// FP64-accurate GEMM on the tcgen05 tensor cores (sm_103a) by error-free
// operand slicing (the Ozaki scheme: Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012).
//
// Every row i of op(A) is scaled by 2^-ea_i (ea_i = exponent of the row's
// largest |entry|, shared by all terms of a grouped sum) and expanded as
// 2^-8 sum_{s=1..7} qa_s 2^-8(s-1) with integers |qa_s| <= 256; likewise every
// column j of op(B) with eb_j.  Each slice q~_s = q_s 2^-8(s-1) is exact in
// BF16.  Then
//   op(A) op(B) = 2^(ea_i + eb_j - 16) sum_{s+t <= 8} A~_s B~_t  (+ O(2^-56) x row/col maxima),
// and every BF16 x BF16 product is exact in FP32.  The 28 slice products are
// issued as tcgen05.mma kind::f16 (BF16 in, FP32 accumulate in TMEM) into six
// accumulators by g = s + t: g = 2, 3, 4, 5, 6 and "g >= 7".  For g <= 6 the
// integer sums of 128 consecutive k stay below 2^24 (|q_1| <= 256, |q_s| <=
// 128 for s >= 2), so those accumulators are exact and are added into FP64
// registers every 128 k.  The g >= 7 accumulator holds terms below 2^-40 of
// the result; its FP32 rounding is far below FP64 rounding, and it is added
// at the end.  The FP64 sum is then scaled by 2^(ea_i + eb_j - 16).
//
// Layout: a CTA computes a 128 x 64 FP64 output tile with 128 threads and
// 6 x 64 TMEM columns (512 allocated).  Per
// 64-wide k chunk it stages 7 A slices (128 x 64) and 7 B slices (64 x 64) in
// shared memory as K-major 8 x 16-byte core matrices (no swizzle), thread 0
// issues the 28 x 4 MMAs (M = 128, N = 64, K = 16), completion is signalled
// through tcgen05.commit on an mbarrier (bounded wait), and the four warps
// read their 32 TMEM lanes each with tcgen05.ld.
#include <cuda_bf16.h>

#include <climits>

#include "tc_gemm.h"

namespace zcsd {

namespace {

constexpr int TC_BM = 128, TC_BN = 64, TC_BK = 32, TC_S = 7;  // TC_BK: k per pipeline stage
constexpr int TC_KALIGN = 64;  // slices are padded along k to the slicing tile
constexpr int TC_THREADS = 256;  // warp w: TMEM lanes 32 (w % 4) .., columns 32 (w / 4) ..
constexpr int TC_CPT = TC_BN / 2;  // output columns per thread
constexpr int TC_NACC = 6;          // accumulators: g = 2..6 exact, g >= 7
constexpr int TC_TMEM_COLS = 512;   // power of two >= TC_NACC * TC_BN + 2 * TC_BN
constexpr int TC_ILO = TC_NACC * TC_BN, TC_IHI = TC_ILO + TC_BN;  // fixed-point sum (low / high words)
constexpr int TC_SLICE_A_BYTES = TC_BM * TC_BK * 2;  // 8 KiB
constexpr int TC_SLICE_B_BYTES = TC_BN * TC_BK * 2;  // 4 KiB
constexpr int TC_STAGE_A = TC_S * TC_SLICE_A_BYTES, TC_STAGE_B = TC_S * TC_SLICE_B_BYTES;
constexpr int TC_SMEM = 2 * (TC_STAGE_A + TC_STAGE_B) + 1024;  // two stages
constexpr long long TC_WAIT_LIMIT = 1LL << 26;
constexpr int TC_MAX_DRAINS = 120;  // intermediate drains before the int64 sum is written out

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ int ceil_div_d(int a, int b) { return (a + b - 1) / b; }

// tcgen05 shared-memory matrix descriptor: start address, leading-dimension
// byte offset (next core matrix along K), stride byte offset (next 8-row group
// along M/N), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

// 16-byte global -> shared copy without a register round trip (both addresses
// are 16-byte aligned: slice rows are padded to multiples of 64 elements)
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(sdst)), "l"(gsrc) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t phase, long long limit = TC_WAIT_LIMIT) {
  uint32_t done = 0;
  for (long long it = 0; it < limit && !done; ++it) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(phase));
  }
  return done != 0;
}

// 16 FP32 columns of this thread's TMEM lane starting at column `col`
__device__ __forceinline__ void tmem_ld16(uint32_t addr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
}

__device__ __forceinline__ void tmem_st16(uint32_t addr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n" ::"r"(addr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]));
  asm volatile("tcgen05.wait::st.sync.aligned;");
}

// The fixed-point sum I = 2^32 sum_{g=2..6} (group g) of 16 columns lives in
// TMEM (low words at column TC_ILO, high words at TC_IHI) between drains, so
// no registers stay live across the k loop.
__device__ __forceinline__ void ifix_load16(uint32_t tmem_row, int c, long long (&I)[16]) {
  uint32_t lo[16], hi[16];
  tmem_ld16(tmem_row + (uint32_t)(TC_ILO + c), lo);
  tmem_ld16(tmem_row + (uint32_t)(TC_IHI + c), hi);
#pragma unroll
  for (int j = 0; j < 16; ++j) I[j] = (long long)(((unsigned long long)hi[j] << 32) | lo[j]);
}

__device__ __forceinline__ void ifix_store16(uint32_t tmem_row, int c, const long long (&I)[16]) {
  uint32_t lo[16], hi[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    lo[j] = (uint32_t)(unsigned long long)I[j];
    hi[j] = (uint32_t)((unsigned long long)I[j] >> 32);
  }
  tmem_st16(tmem_row + (uint32_t)(TC_ILO + c), lo);
  tmem_st16(tmem_row + (uint32_t)(TC_IHI + c), hi);
}

// Exact groups g = 2..6 (accumulators a = g - 2) into I: accumulator a holds
// an integer multiple of 2^-8a below 2^24 in magnitude (exact in FP32), so
// x 2^8a and a conversion give that integer exactly, which enters I shifted
// left by 8 (4 - a).  Integer arithmetic only: the FP64 pipe runs 2 lanes per
// clock per SM.
__device__ __forceinline__ void drain_exact16(uint32_t tmem_row, int c, long long (&I)[16]) {
#pragma unroll
  for (int a = 0; a < TC_NACC - 1; ++a) {
    uint32_t r[16];
    tmem_ld16(tmem_row + (uint32_t)(a * TC_BN + c), r);
    const float up = __int_as_float((127 + 8 * a) << 23);  // 2^(8a)
#pragma unroll
    for (int j = 0; j < 16; ++j) I[j] += (long long)__float2int_rn(__uint_as_float(r[j]) * up) << (8 * (4 - a));
  }
}

// J 2^e as a double, rounded to nearest (ties to even on J's bits), built with
// integer instructions: GB300's FP64 pipe retires 2 lanes per clock per SM,
// so the epilogue keeps FP64 work to the beta C term.  Results outside the
// normal range take ldexp.
__device__ __forceinline__ double fix_to_double(long long J, int e) {
  if (J == 0) return 0.0;
  const unsigned long long sgn = J < 0 ? (1ull << 63) : 0ull;
  const unsigned long long mag = J < 0 ? 0ull - (unsigned long long)J : (unsigned long long)J;
  const int lz = __clzll((long long)mag);
  const unsigned long long m = mag << lz;  // bit 63 set: J = m 2^-lz
  unsigned long long mant = m >> 11;       // 53 bits with the leading one
  const unsigned long long rem = m & 0x7FFull;
  int E = 63 - lz + e;
  if (rem > 0x400ull || (rem == 0x400ull && (mant & 1ull))) {
    ++mant;
    if (mant >> 53) {
      mant >>= 1;
      ++E;
    }
  }
  if (E < -1022 || E > 1023) return ldexp((double)J, e);
  return __longlong_as_double((long long)(sgn | ((unsigned long long)(E + 1023) << 52) | (mant & 0xFFFFFFFFFFFFFull)));
}

// d 2^e alpha: the power of two is built from its bits when it is a normal
// number, with the sign of alpha folded in when |alpha| = 1 (asgn = sign bit)
__device__ __forceinline__ double scale_out(double d, int e, double alpha, bool unit, unsigned long long asgn) {
  if (e >= -1022 && e <= 1023) {
    const double v = d * __longlong_as_double((long long)(((unsigned long long)(e + 1023) << 52) | asgn));
    return unit ? v : alpha * v;
  }
  return alpha * ldexp(d, e);
}

struct TcArgs {
  int m, n, kpad, nsum, batch;
  const __nv_bfloat16* Asl;  // [batch][nsum][S][mpad][kpad]
  const __nv_bfloat16* Bsl;  // [batch][nsum][S][npad][kpad]
  const int* ea;             // [batch][mpad]
  const int* eb;             // [batch][npad]
  long long sAsl, sBsl;      // elements per (batch, term) slice set
  int mpad, npad;
  int kb_flags;              // K_FROM_COL / K_FROM_ROW / K_TO_COL / K_TO_ROW
  int ksplit;                // split-K parts: problem b, part s writes C_{b * ksplit + s}
  int uplo;
  double alpha, beta;
  const double* Cin; int ldcin; long long sCin; int bdivC;
  double* C; int ldc; long long sC;
  int* err;
  int max_drains;          // drains between write-outs of the int64 sum
  long long probe_wait;    // > 0: first poll a barrier nothing signals (timeout-path tests)
};

__global__ void __launch_bounds__(TC_THREADS, 1) tc_gemm_kernel(TcArgs g) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1 KiB alignment of the operand area
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = smem;
  unsigned char* sB = smem + 2 * TC_STAGE_A;
  __shared__ __align__(8) uint64_t mbar[3];  // MMA completion of the stage in buffer 0 / 1; [2]: probe
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int z = blockIdx.z;
  const int b = z / g.ksplit, kpart = z % g.ksplit;
  const int m0 = blockIdx.x * TC_BM, n0 = blockIdx.y * TC_BN;
  if (g.uplo == 1 && m0 > n0 + TC_BN - 1) return;
  if (g.uplo == 2 && n0 > m0 + TC_BM - 1) return;
  int kb = 0, ke = g.kpad;
  if (g.ksplit > 1) {  // split-K: part kpart takes one 64-aligned K range
    const int kc = ceil_div_d(ceil_div_d(g.kpad, g.ksplit), TC_BK) * TC_BK;
    kb = kpart * kc;
    ke = min(g.kpad, kb + kc);
  }
  if (g.kb_flags & K_FROM_COL) kb = max(kb, n0);
  if (g.kb_flags & K_FROM_ROW) kb = max(kb, m0);
  if (g.kb_flags & K_TO_COL) ke = min(ke, n0 + TC_BN);
  if (g.kb_flags & K_TO_ROW) ke = min(ke, m0 + TC_BM);
  kb = (kb / TC_BK) * TC_BK;

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[0])), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[1])), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[2])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(TC_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  const uint32_t tmem_row = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)((warp >> 2) * TC_CPT);
  const int cbase = n0 + (warp >> 2) * TC_CPT;  // first output column of this thread
  constexpr uint32_t IDESC = idesc_bf16(TC_BM, TC_BN);
  const uint32_t mbar_addr[2] = {smem_u32(&mbar[0]), smem_u32(&mbar[1])};

  {  // fixed-point sum I = 0
    const long long z16[16] = {};
#pragma unroll
    for (int c = 0; c < TC_CPT; c += 16) ifix_store16(tmem_row, c, z16);
  }
  bool ok = true;
  if (g.probe_wait > 0) {
    // test hook: a bounded wait on a barrier that nothing signals, before
    // any copy or MMA is issued; it runs out and the launch takes the
    // timeout path (NaN outputs, error flag)
    ok = __syncthreads_and(tid != 0 || mbar_wait(smem_u32(&mbar[2]), 0u, g.probe_wait)) != 0;
  }
  // accumulator a at TMEM columns [64 a, 64 a + 64): a = g - 2 for g <= 6, a = 5 for g >= 7
  uint32_t filled = 0;  // bit a set: accumulator a holds data since its last drain
  int chunks_since_drain = 0, nchunks = 0, ndrain = 0;
  bool flushed = false;  // a partial sum was already written to C
  const int row = m0 + (warp & 3) * 32 + lane;
  const int ea = row < g.m ? g.ea[(long long)b * g.mpad + row] : 0;
  const bool aunit = g.alpha == 1.0 || g.alpha == -1.0;
  const unsigned long long asgn = (aunit && g.alpha < 0.0) ? (1ull << 63) : 0ull;
  double* C = g.C + (long long)z * g.sC;
  const double* Cin = (g.Cin && kpart == 0 && g.beta != 0.0) ? g.Cin + (long long)(b / g.bdivC) * g.sCin : nullptr;

  // stages q = 0 .. Q-1: term js = q / nst, k range [kb + 32 (q % nst), +32);
  // the slices of stage q + 1 load (cp.async) into the other buffer while
  // the MMAs of stage q run; a buffer is refilled once the MMAs that read it
  // have signalled their mbarrier
  const int nst = ke > kb ? (ke - kb + TC_BK - 1) / TC_BK : 0;
  const int Q = g.nsum * nst;
  auto load_stage = [&](int q, int buf) {
    const int js = q / nst, k0 = kb + (q % nst) * TC_BK;
    const __nv_bfloat16* Ab = g.Asl + ((long long)b * g.nsum + js) * g.sAsl;
    const __nv_bfloat16* Bb = g.Bsl + ((long long)b * g.nsum + js) * g.sBsl;
    unsigned char* dA = sA + buf * TC_STAGE_A;
    unsigned char* dB = sB + buf * TC_STAGE_B;
    // vector v = (slice, row, k/8): 16 bytes of 8 consecutive k, placed as
    // K-major 8 x 16-byte core matrices
    for (int v = tid; v < TC_S * TC_BM * (TC_BK / 8); v += TC_THREADS) {
      const int sl = v / (TC_BM * (TC_BK / 8)), rem = v % (TC_BM * (TC_BK / 8));
      const int r = rem / (TC_BK / 8), kq = rem % (TC_BK / 8);
      cp_async16(dA + sl * TC_SLICE_A_BYTES + ((r >> 3) * (TC_BK / 8) + kq) * 128 + (r & 7) * 16,
                 Ab + (long long)sl * g.mpad * g.kpad + (long long)(m0 + r) * g.kpad + k0 + kq * 8);
    }
    for (int v = tid; v < TC_S * TC_BN * (TC_BK / 8); v += TC_THREADS) {
      const int sl = v / (TC_BN * (TC_BK / 8)), rem = v % (TC_BN * (TC_BK / 8));
      const int r = rem / (TC_BK / 8), kq = rem % (TC_BK / 8);
      cp_async16(dB + sl * TC_SLICE_B_BYTES + ((r >> 3) * (TC_BK / 8) + kq) * 128 + (r & 7) * 16,
                 Bb + (long long)sl * g.npad * g.kpad + (long long)(n0 + r) * g.kpad + k0 + kq * 8);
    }
    asm volatile("cp.async.commit_group;");
  };
  uint32_t ph[2] = {0u, 0u};
  bool pend[2] = {false, false};
  // wait (bounded, uniform over the CTA) for the MMAs committed on buffer bf
  auto wait_buf = [&](int bf) {
    if (!pend[bf]) return;
    ok = __syncthreads_and(ok && mbar_wait(mbar_addr[bf], ph[bf])) != 0;
    ph[bf] ^= 1u;
    pend[bf] = false;
  };
  if (Q > 0) load_stage(0, 0);
  for (int q = 0; q < Q && ok; ++q) {
    const int buf = q & 1;
    asm volatile("cp.async.wait_group 0;" ::: "memory");  // stage q (the only group in flight)
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a0 = smem_u32(sA + buf * TC_STAGE_A), b0 = smem_u32(sB + buf * TC_STAGE_B);
      for (int s1 = 1; s1 <= TC_S; ++s1)
        for (int t1 = 1; t1 <= TC_S + 1 - s1; ++t1) {
          const int gi = s1 + t1;
          const int a = gi <= 6 ? gi - 2 : 5;
#pragma unroll
          for (int ks = 0; ks < TC_BK / 16; ++ks) {
            const uint64_t ad = smem_desc(a0 + (s1 - 1) * TC_SLICE_A_BYTES + ks * 256, 128, (TC_BK / 8) * 128);
            const uint64_t bd = smem_desc(b0 + (t1 - 1) * TC_SLICE_B_BYTES + ks * 256, 128, (TC_BK / 8) * 128);
            const uint32_t accum = (filled >> a) & 1u;
            mma_bf16(tmem + (uint32_t)(a * TC_BN), ad, bd, IDESC, accum);
            filled |= (1u << a);
          }
        }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          mbar_addr[buf]));
    }
    pend[buf] = true;
    ++chunks_since_drain;
    ++nchunks;
    const bool last = q + 1 == Q;
    if (!last) {  // prefetch stage q + 1 once the MMAs of stage q - 1 released its buffer
      wait_buf(buf ^ 1);
      if (ok) load_stage(q + 1, buf ^ 1);
    }
    // intermediate drain of the exact groups every 128 k (the final one is
    // below); every stage writes all six accumulators, so a drain is always
    // followed by fresh MMAs
    if (ok && !last && chunks_since_drain * TC_BK >= 128) {
      wait_buf(buf);  // all MMAs so far complete
      asm volatile("tcgen05.fence::after_thread_sync;");
      if (ok) {
        // |I| grows by < 2^56.1 per drain: every TC_MAX_DRAINS drains the
        // partial sum is written out before it can leave int64 (K > ~15k)
        const bool flush = ++ndrain == g.max_drains;
#pragma unroll
        for (int c = 0; c < TC_CPT; c += 16) {
          long long I[16];
          ifix_load16(tmem_row, c, I);
          drain_exact16(tmem_row, c, I);
          if (flush) {
            if (row < g.m)
#pragma unroll
              for (int j = 0; j < 16; ++j) {
                const int col = cbase + c + j;
                if (col < g.n) {
                  double v = scale_out((double)I[j], ea + g.eb[(long long)b * g.npad + col] - 48, g.alpha, aunit, asgn);
                  const long long ic = row + (long long)col * g.ldc;
                  if (flushed) v += C[ic];
                  else if (Cin) v = fma(g.beta, Cin[row + (long long)col * g.ldcin], v);
                  C[ic] = v;
                }
              }
#pragma unroll
            for (int j = 0; j < 16; ++j) I[j] = 0;
          }
          ifix_store16(tmem_row, c, I);
        }
        if (flush) {
          flushed = true;
          ndrain = 0;
        }
        if (tid == 0) filled &= (1u << (TC_NACC - 1));  // g >= 7 keeps running
        chunks_since_drain = 0;
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();  // TMEM read before the next MMAs
    }
  }
  // the last stage's MMAs (and any other pending commit)
  wait_buf(0);
  wait_buf(1);
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (!ok && lane == 0) atomicExch(g.err, 1);
  // ---- final drain + epilogue, 16 columns at a time (row = this thread's
  // TMEM lane): value = (I + 2^32 acc_{g>=7}) 2^(ea + eb - 48), then alpha,
  // beta; about five FP64 operations per output
  const bool have = ok && nchunks > 0;
#pragma unroll
  for (int c0 = 0; c0 < TC_CPT; c0 += 16) {
    uint32_t r7[16];
    long long I[16];
    ifix_load16(tmem_row, c0, I);
    if (have) {
      drain_exact16(tmem_row, c0, I);
      tmem_ld16(tmem_row + (uint32_t)((TC_NACC - 1) * TC_BN + c0), r7);
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) r7[j] = 0u;
    }
    if (row < g.m) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int col = cbase + c0 + j;
        if (col < g.n) {
          // (I + 2^32 acc7) 2^(ea + eb - 48): while |I| < 2^55, I 2^8 plus
          // acc7 rounded at 2^-40 stays exact to 2^-57 of the operands'
          // row x column maxima; above, acc7 rounded at 2^-32 is below 2^-56
          // of the result
          long long J = I[j];
          int e = ea + g.eb[(long long)b * g.npad + col] - 48;
          const float a7 = __uint_as_float(r7[j]);
          const bool fine = J > -(1LL << 55) && J < (1LL << 55);
          const float t = a7 * (fine ? 0x1p40f : 0x1p32f);
          const long long add = fabsf(t) < 2147483648.0f ? (long long)__float2int_rn(t) : __float2ll_rn(t);
          if (fine) {
            J = J * 256 + add;
            e -= 8;
          } else {
            J += add;
          }
          double v = fix_to_double(J, e);
          if (aunit) v = __longlong_as_double(__double_as_longlong(v) ^ (long long)asgn);
          else v *= g.alpha;
          const long long ic = row + (long long)col * g.ldc;
          if (flushed) v += C[ic];
          else if (Cin) v = fma(g.beta, Cin[row + (long long)col * g.ldcin], v);
          C[ic] = ok ? v : NAN;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
}

// ---- slicing: exponents of rows of op(A) (cols of op(B)) then the 7 slices

// Slicing works on 64 x 64 tiles of op(X_{b,j}) staged in shared memory, so
// that global reads follow the memory order of X (op N: i fastest, op T: k
// fastest) and the slice writes follow the [i][k] (k fastest) order.
constexpr int SL_T = 64;

__device__ __forceinline__ void load_tile(double (*tile)[SL_T + 1], const double* X, int ld, int op, int rows, int K,
                                          int i0, int k0, double wj, const int* ek, int sgn) {
  for (int e = threadIdx.x; e < SL_T * SL_T; e += blockDim.x) {
    // a = fastest index in memory, c = the other
    const int a = e % SL_T, c = e / SL_T;
    int i, k;
    if (op == OP_N) { i = i0 + a; k = k0 + c; }
    else { k = k0 + a; i = i0 + c; }
    double v = 0.0;
    if (i < rows && k < K) {
      v = wj * (op == OP_N ? X[i + (long long)k * ld] : X[k + (long long)i * ld]);
      if (ek) {  // inner-dimension balance: x 2^(sgn e_k), exact (sentinel e_k: zero row of op(B), no shift)
        const int sh = ek[k] < -2000 ? 0 : sgn * ek[k];
        v = (sh >= -1022 && sh <= 1023) ? v * __longlong_as_double((long long)(sh + 1023) << 52) : ldexp(v, sh);
      }
    }
    tile[i - i0][k - k0] = v;
  }
}

// exponent e_i with max |x| < 2^e_i over row i of w_j op(X_{b,j}), all terms j
__global__ void tc_row_exp_kernel(int rows, int K, int nsum, int op, const double* X, int ld, long long sX,
                                  long long sXj, int bdiv, const double* w, int rpad, int* e, const int* ek,
                                  int ekpad, int sgn) {
  __shared__ double tile[SL_T][SL_T + 1];
  const int i0 = blockIdx.x * SL_T, k0 = blockIdx.y * SL_T;
  const int b = blockIdx.z / nsum, js = blockIdx.z % nsum;
  load_tile(tile, X + (long long)(b / bdiv) * sX + js * sXj, ld, op, rows, K, i0, k0, w[js],
            ek ? ek + (long long)b * ekpad : nullptr, sgn);
  __syncthreads();
  // 4 threads per row, then one atomic per row of the tile.  The exponent
  // is read from the bits: a normal |x| lies in [2^(E-1023), 2^(E-1022)) for
  // biased exponent E, so E - 1022 bounds it (frexp's exponent); zeros and
  // subnormals (E = 0) do not raise the row maximum.
  const int r = threadIdx.x / 4, q = threadIdx.x % 4;
  int ex = INT_MIN;
  for (int k = q; k < SL_T; k += 4) {
    const int E = (int)((__double_as_longlong(tile[r][k]) >> 52) & 0x7FF);
    if (E > 0) ex = max(ex, E - 1022);
  }
  ex = max(ex, __shfl_xor_sync(0xffffffffu, ex, 1));
  ex = max(ex, __shfl_xor_sync(0xffffffffu, ex, 2));
  if (q == 0 && ex != INT_MIN && i0 + r < rows) atomicMax(&e[(long long)b * rpad + i0 + r], ex);
}

// slices q~_s (s = 1..7) of w_j op(X_{b,j}) 2^-e_i, stored [b][j][s][i][kpad]
__global__ void tc_slice_kernel(int rows, int K, int nsum, int op, const double* X, int ld, long long sX, long long sXj,
                                int bdiv, const double* w, const int* e, int rpad, int kpad, __nv_bfloat16* out,
                                long long sOut, const int* ek, int sgn) {
  __shared__ double tile[SL_T][SL_T + 1];
  const int i0 = blockIdx.x * SL_T, k0 = blockIdx.y * SL_T;
  const int b = blockIdx.z / nsum, js = blockIdx.z % nsum;
  load_tile(tile, X + (long long)(b / bdiv) * sX + js * sXj, ld, op, rows, K, i0, k0, w[js],
            ek ? ek + (long long)b * kpad : nullptr, sgn);
  __syncthreads();
  __nv_bfloat16* o = out + ((long long)b * nsum + js) * sOut;
  for (int t = threadIdx.x; t < SL_T * SL_T; t += blockDim.x) {
    const int kk = t % SL_T, ii = t / SL_T;
    const int i = i0 + ii, k = k0 + kk;
    if (i >= rpad || k >= kpad) continue;
    // X = round(x 2^(56 - e_i)) as a 64-bit integer (|X| <= 2^56), then its
    // balanced base-256 digits from the bottom: d = ((X + 128) mod 256) - 128,
    // X <- (X - d) / 256; the top digit q_1 keeps |q_1| <= 256, the others
    // |q_s| <= 128.  Two FP64 multiplies and one conversion per element; the
    // rest is integer arithmetic.
    long long X = 0;
    const int ei = (i < rows) ? e[(long long)b * rpad + i] : INT_MIN;
    if (ei > -2000 && tile[ii][kk] != 0.0) {  // rows without a nonzero entry keep the sentinel exponent
      const double v = tile[ii][kk];
      const int sh = 56 - ei;  // in [-968, 1130] for finite nonzero data
      // 2^sh as two exact, normal powers of two
      const int s1 = sh / 2, s2 = sh - s1;
      X = __double2ll_rn(v * __longlong_as_double((long long)(1023 + s1) << 52) *
                         __longlong_as_double((long long)(1023 + s2) << 52));
    }
    int q[TC_S];
#pragma unroll
    for (int sidx = TC_S - 1; sidx >= 1; --sidx) {
      const int d = (int)((X + 128) & 255) - 128;
      q[sidx] = d;
      X = (X - d) >> 8;
    }
    q[0] = (int)X;
#pragma unroll
    for (int sidx = 0; sidx < TC_S; ++sidx)
      o[(long long)sidx * rpad * kpad + (long long)i * kpad + k] =
          __float2bfloat16_rn((float)q[sidx] * __int_as_float((127 - 8 * sidx) << 23));
  }
}


}  // namespace

thread_local TcState t_tc;

bool tc_gemm_supported(const GemmArgs<double>& g) {
  return g.ksplit >= 1 && g.m >= 1 && g.n >= 1 && g.k >= 1 && g.nsum >= 1;
}

int tc_pick_ksplit(const GemmArgs<double>& g, int cap) {
  // one CTA per SM (shared memory and TMEM): aim at one full wave of 152
  // CTAs, with at least 4 k chunks (256 k) per part
  const long long tiles = (long long)ceil_div(g.m, TC_BM) * ceil_div(g.n, TC_BN) * g.batch;
  if (tiles >= 152) return 1;
  const int s = (int)std::min<long long>({(long long)cap, (152 + tiles - 1) / tiles, (long long)std::max(1, g.k / 256)});
  return std::max(1, s);
}

bool tc_will_handle(const GemmArgs<double>& g) {
  // The tile is 128 x 64 with a 64-wide k chunk: products with a short side
  // (m < 128, n < 64 or k < 64) stay on the FP64 pipe.
  return t_tc.enabled && t_tc.ar && ((t_tc.sites >> g.site) & 1u) && tc_gemm_supported(g) && g.m >= TC_BM &&
         g.n >= TC_BN && g.k >= 64;
}

void tc_gemm(const GemmArgs<double>& g, cudaStream_t st, Arena& ar, int* err) {
  ProfToken tok = prof_begin(st);  // slicing + tensor-core kernel
  const int mpad = ceil_div(g.m, TC_BM) * TC_BM;
  const int npad = ceil_div(g.n, TC_BN) * TC_BN;
  const int kpad = ceil_div(g.k, TC_KALIGN) * TC_KALIGN;
  const int nsum = std::max(g.nsum, 1);
  const size_t mk = ar.mark();
  // op(A) and op(B)^T the same matrix (a Gram product Y^* Y): one set of
  // slices and exponents serves both operands
  bool same = g.A == g.B && g.lda == g.ldb && g.sA == g.sB && g.sAj == g.sBj && g.bdivA == g.bdivB && g.m == g.n &&
              ((g.opA != OP_N) == (g.opB == OP_N));
  for (int j = 0; j < nsum && same; ++j) same = g.w[j] == 1.0;
  const long long sAsl = (long long)TC_S * mpad * kpad, sBsl = same ? sAsl : (long long)TC_S * npad * kpad;
  __nv_bfloat16* Asl = ar.get<__nv_bfloat16>((size_t)sAsl * nsum * g.batch);
  __nv_bfloat16* Bsl = same ? Asl : ar.get<__nv_bfloat16>((size_t)sBsl * nsum * g.batch);
  int* ea = ar.get<int>((size_t)mpad * g.batch);
  int* eb = same ? ea : ar.get<int>((size_t)npad * g.batch);
  double* w = ar.get<double>(2 * MAX_SUM);
  // host weights -> device (term weights apply to A; B gets unit weights)
  double hw[2 * MAX_SUM];
  for (int j = 0; j < MAX_SUM; ++j) { hw[j] = g.w[j]; hw[MAX_SUM + j] = 1.0; }
  ZCSD_CUDA(cudaMemcpyAsync(w, hw, sizeof(hw), cudaMemcpyHostToDevice, st));
  // 0xC0C0C0C0 = -1061109568: "no nonzero entry"; two of them still add up
  // without overflow, and such rows/columns have all-zero slices
  ZCSD_CUDA(cudaMemsetAsync(ea, 0xC0, sizeof(int) * mpad * g.batch, st));
  if (!same) ZCSD_CUDA(cudaMemsetAsync(eb, 0xC0, sizeof(int) * npad * g.batch, st));
  // op(A): rows = m, K = k;  op(B)^T: rows = n, K = k  (op(B)^T = B^T for op N, B for op T)
  // real data: conjugate-transpose is the transpose
  const int opA = (g.opA == OP_N) ? OP_N : OP_T;
  const int opBt = (g.opB == OP_N) ? OP_T : OP_N;
  const dim3 ga(mpad / SL_T, kpad / SL_T, g.batch * nsum), gb(npad / SL_T, kpad / SL_T, g.batch * nsum);
  // inner-dimension balance (one term only): e_k bounds row k of op(B);
  // op(A) D and D^-1 op(B) with D = diag(2^e_k) have the same product, and
  // per-row / per-column slicing of the balanced operands is accurate
  // relative to max_k |a_ik| |b_k.| instead of max |a_i.| max |b_.j|
  int* ek = nullptr;
  if (g.kbal && nsum == 1 && !same) {
    ek = ar.get<int>((size_t)kpad * g.batch);
    ZCSD_CUDA(cudaMemsetAsync(ek, 0xC0, sizeof(int) * kpad * g.batch, st));
    const dim3 gk(kpad / SL_T, ceil_div(g.n, SL_T), g.batch);
    tc_row_exp_kernel<<<gk, 256, 0, st>>>(g.k, g.n, 1, g.opB == OP_N ? OP_N : OP_T, g.B, g.ldb, g.sB, 0, g.bdivB,
                                          w + MAX_SUM, kpad, ek, nullptr, 0, 0);
    ZCSD_LAUNCH();
  }
  tc_row_exp_kernel<<<ga, 256, 0, st>>>(g.m, g.k, nsum, opA, g.A, g.lda, g.sA, g.sAj, g.bdivA, w, mpad, ea, ek, kpad,
                                        1);
  ZCSD_LAUNCH();
  if (!same) {
    tc_row_exp_kernel<<<gb, 256, 0, st>>>(g.n, g.k, nsum, opBt, g.B, g.ldb, g.sB, g.sBj, g.bdivB, w + MAX_SUM, npad,
                                          eb, ek, kpad, -1);
    ZCSD_LAUNCH();
  }
  tc_slice_kernel<<<ga, 256, 0, st>>>(g.m, g.k, nsum, opA, g.A, g.lda, g.sA, g.sAj, g.bdivA, w, ea, mpad, kpad, Asl,
                                      sAsl, ek, 1);
  ZCSD_LAUNCH();
  if (!same) {
    tc_slice_kernel<<<gb, 256, 0, st>>>(g.n, g.k, nsum, opBt, g.B, g.ldb, g.sB, g.sBj, g.bdivB, w + MAX_SUM, eb, npad,
                                        kpad, Bsl, sBsl, ek, -1);
    ZCSD_LAUNCH();
  }
  TcArgs t;
  t.m = g.m; t.n = g.n; t.kpad = kpad; t.nsum = nsum; t.batch = g.batch;
  t.Asl = Asl; t.Bsl = Bsl; t.ea = ea; t.eb = eb; t.sAsl = sAsl; t.sBsl = sBsl; t.mpad = mpad;
  t.npad = same ? mpad : npad;  // row pitch of the B slices and exponents
  t.kb_flags = g.kflags; t.ksplit = std::max(1, g.ksplit); t.uplo = g.uplo; t.alpha = re(g.alpha); t.beta = re(g.beta);
  t.Cin = g.Cin; t.ldcin = g.ldcin; t.sCin = g.sCin; t.bdivC = g.bdivC;
  t.C = g.C; t.ldc = g.ldc; t.sC = g.sC; t.err = err;
  t.max_drains = t_tc.flush_every > 0 ? std::min(t_tc.flush_every, TC_MAX_DRAINS) : TC_MAX_DRAINS;
  t.probe_wait = t_tc.probe_wait;
  ZCSD_CUDA(cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
  dim3 grid(mpad / TC_BM, npad / TC_BN, g.batch * t.ksplit);
  tc_gemm_kernel<<<grid, TC_THREADS, TC_SMEM, st>>>(t);
  ZCSD_LAUNCH();
  if (tok.slot >= 0) {
    // FP64-equivalent multiply-add work over the tiles executed
    double fma = 0.0;
    for (int bx = 0; bx < mpad / TC_BM; ++bx)
      for (int by = 0; by < npad / TC_BN; ++by) {
        const int m0 = bx * TC_BM, n0 = by * TC_BN;
        if (g.uplo == 1 && m0 > n0 + TC_BN - 1) continue;
        if (g.uplo == 2 && n0 > m0 + TC_BM - 1) continue;
        int kb = 0, ke = g.k;
        if (g.kflags & K_FROM_COL) kb = std::max(kb, n0);
        if (g.kflags & K_FROM_ROW) kb = std::max(kb, m0);
        if (g.kflags & K_TO_COL) ke = std::min(ke, n0 + TC_BN);
        if (g.kflags & K_TO_ROW) ke = std::min(ke, m0 + TC_BM);
        if (ke > kb)
          fma += (double)std::min(TC_BM, g.m - m0) * std::min(TC_BN, g.n - n0) * (ke - kb);
      }
    prof_end(tok, st, PK_TC, 2.0 * fma * nsum * g.batch, g.site);
  }
  ar.release(mk);
}

}  // namespace zcsd
