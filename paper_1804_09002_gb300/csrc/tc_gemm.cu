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
// and every BF16 x BF16 product is exact in FP32.  The 28 slice products
// accumulate by g = s + t into seven FP32 accumulators in TMEM (g = 2..8).
// For g <= 6 the integer sums of 128 consecutive k stay below 2^24
// (|q_1| <= 256, |q_s| <= 128 for s >= 2), so those accumulators are exact;
// every 128 k they are converted to a 64-bit fixed-point sum kept in
// registers and zeroed.  Groups 7 and 8 hold terms below 2^-40 of the result
// and are read once at the end.
//
// Kernel organisation (one CTA per SM, persistent over output tiles):
//  * warp 0, one lane: producer.  Per 16-wide k stage it loads the 7 A slices
//    (128 rows) and the 7 B slices (64 rows) with one cp.async.bulk.tensor
//    (TMA) box each into a 5-deep ring of stages (full/empty mbarriers).
//    The slices are stored in global memory as [term][k/8][slice][row][8 k],
//    so each box lands as K-major 8 x 16-byte core matrices with the rows of
//    all 7 slices consecutive;
//  * warp 1, one lane: MMA issuer.  Because the B rows of slices t = 1..7
//    are consecutive and accumulator g sits at TMEM columns 64 (g - 2), the
//    products of A slice s with every B slice t <= 8 - s form ONE product of
//    N = 64 (8 - s) columns into accumulators g = s + 1 .. 8: ten MMAs
//    (M = 128, N <= 256, K = 16) per stage instead of 28;
//  * warps 2..17: epilogue.  Warp w reads TMEM lanes 32 (w mod 4) .. (its
//    output rows) and one quarter of the 64 columns; it drains the exact
//    accumulators every 128 k, and at the end of a tile builds the FP64
//    result from the int64 sum and writes C.
// Every wait is bounded; a wait that runs out sets the CTA's abort flag and
// the device error flag, every role leaves its loop, the producer waits
// (bounded) for its copies in flight and the MMA issuer for its MMAs before
// TMEM is released, and the outputs of unfinished tiles are NaN.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <climits>
#include <mutex>

#include "tc_gemm.h"

namespace zcsd {

namespace {

constexpr int TC_BM = 128, TC_BN = 64;
constexpr int TC_SMAX = 7;           // slices of an FP64-accurate product
constexpr int TC_KS = 16;            // k per pipeline stage (one MMA K)
constexpr int TC_KALIGN = 64;        // slices are padded along k to the slicing tile
constexpr int TC_DRAIN_STAGES = 128 / TC_KS;
constexpr int TC_EPI_WARPS = 16;
constexpr int TC_THREADS = 32 * (2 + TC_EPI_WARPS);
constexpr int TC_CPT = TC_BN / 4;    // output columns per epilogue thread (16)
constexpr int TC_TMEM_COLS = 512;    // power of two >= 7 x 64
constexpr long long TC_WAIT_LIMIT = 1LL << 26;
constexpr int TC_MAX_DRAINS = 120;  // intermediate drains before the int64 sum is written out

// Layout constants of a product with S slices per operand (S = 5, 6, 7:
// 40, 48 or 56 bits): S(S + 1) / 2 slice products into S accumulators
// (g = 2 .. S + 1); g <= 6 are exact and drained every 128 k.
template <int S>
struct TcCfg {
  static constexpr int NACC = S;
  static constexpr int NEXACT = S < 5 ? S : 5;
  static constexpr int A_STAGE = S * TC_BM * TC_KS * 2;  // 28 KiB at S = 7
  static constexpr int B_STAGE = S * TC_BN * TC_KS * 2;  // 14 KiB at S = 7
  static constexpr int STAGE = A_STAGE + B_STAGE;
  static constexpr int NSTAGE = (225 * 1024) / STAGE < 8 ? (225 * 1024) / STAGE : 8;  // depth of the ring
  static constexpr int SMEM = NSTAGE * STAGE + 1024;
  static constexpr uint32_t LBO_A = S * TC_BM * 16;  // next 8-wide k group
  static constexpr uint32_t LBO_B = S * TC_BN * 16;
  static_assert(SMEM <= 227 * 1024, "stage ring exceeds shared memory");
  static_assert(NACC * TC_BN <= TC_TMEM_COLS, "accumulators exceed TMEM");
  static_assert(S >= 5 && S <= TC_SMAX, "5 to 7 slices");
};
constexpr int TC_NSTAGE_MAX = 8;

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

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, 1, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(ad), "l"(bd), "r"(idesc));
}

__device__ __forceinline__ void mbar_init(uint32_t addr, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count));
}

__device__ __forceinline__ bool mbar_try(uint32_t addr, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(addr), "r"(parity)
      : "memory");
  return done != 0;
}

// Bounded wait for the phase of `parity`; gives up after `limit` polls or
// as soon as the CTA's abort flag is set.  Returns true on completion.
__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity, volatile int* abort_flag,
                                          long long limit = TC_WAIT_LIMIT) {
  for (long long it = 0; it < limit; ++it) {
    if (mbar_try(addr, parity)) return true;
    if (abort_flag && *abort_flag) return false;
  }
  return false;
}

__device__ __forceinline__ void mbar_arrive(uint32_t addr) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(addr) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t addr, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(addr), "r"(bytes) : "memory");
}

// 5-D tiled TMA load into shared memory, completion counted on `mbar`
__device__ __forceinline__ void tma_load5(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3, int c4,
                                          uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
      "%6}], [%7];" ::"r"(dst),
      "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(mbar)
      : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t addr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t addr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 16 zero columns of this thread's TMEM lane starting at `addr`
__device__ __forceinline__ void tmem_zero16(uint32_t addr) {
  const uint32_t z = 0u;
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};\n" ::"r"(addr),
      "r"(z)
      : "memory");
}

// Exact groups g = 2..6 (accumulators a = g - 2) into I: accumulator a holds
// an integer multiple of 2^-8a below 2^24 in magnitude (exact in FP32), so
// x 2^8a and a conversion give that integer exactly, which enters I shifted
// left by 8 (4 - a).  Integer arithmetic only: the FP64 pipe runs 2 lanes per
// clock per SM.
template <int NEXACT>
__device__ __forceinline__ void drain_exact(uint32_t tmem_row, long long (&I)[TC_CPT]) {
#pragma unroll
  for (int a = 0; a < NEXACT; ++a) {
    uint32_t r[TC_CPT];
    tmem_ld16(tmem_row + (uint32_t)(a * TC_BN), r);
    const float up = __int_as_float((127 + 8 * a) << 23);  // 2^(8a)
#pragma unroll
    for (int j = 0; j < TC_CPT; ++j) I[j] += (long long)__float2int_rn(__uint_as_float(r[j]) * up) << (8 * (4 - a));
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

struct TcArgs {
  int m, n, kpad, nsum, batch;
  const int* ea;             // [batch][mpad]
  const int* eb;             // [batch][npad]
  int mpad, npad;            // row pitch of the A / B slices and exponents
  int tiles_n;               // output tiles along n
  int kb_flags;              // K_FROM_COL / K_FROM_ROW / K_TO_COL / K_TO_ROW
  int ksplit;                // split-K parts: problem b, part s writes C_{b * ksplit + s}
  int uplo;
  double alpha, beta;
  const double* Cin; int ldcin; long long sCin; int bdivC;
  double* C; int ldc; long long sC;
  int* err;
  int es;                  // element stride of C and Cin in doubles (2: one part of complex data)
  int max_drains;          // drains between write-outs of the int64 sum
  long long probe_wait;    // > 0: first poll a barrier nothing signals (timeout-path tests)
};

// One output tile of one problem (and split-K part) with its k range.
struct TcItem {
  int m0, n0, b, kpart, kb, nst;  // nst: 16-wide k stages per term
  bool skip;
};

__device__ __forceinline__ TcItem tc_item(const TcArgs& g, int it) {
  TcItem t;
  const int tm = g.mpad / TC_BM, tn = g.tiles_n;
  const int mt = it % tm, nt = (it / tm) % tn, z = it / (tm * tn);
  t.b = z / g.ksplit;
  t.kpart = z % g.ksplit;
  t.m0 = mt * TC_BM;
  t.n0 = nt * TC_BN;
  t.skip = (g.uplo == 1 && t.m0 > t.n0 + TC_BN - 1) || (g.uplo == 2 && t.n0 > t.m0 + TC_BM - 1);
  int kb = 0, ke = g.kpad;
  if (g.ksplit > 1) {  // split-K: part kpart takes one TC_KS-aligned K range
    const int kc = ceil_div_d(ceil_div_d(g.kpad, g.ksplit), TC_KS) * TC_KS;
    kb = t.kpart * kc;
    ke = min(g.kpad, kb + kc);
  }
  if (g.kb_flags & K_FROM_COL) kb = max(kb, t.n0);
  if (g.kb_flags & K_FROM_ROW) kb = max(kb, t.m0);
  if (g.kb_flags & K_TO_COL) ke = min(ke, t.n0 + TC_BN);
  if (g.kb_flags & K_TO_ROW) ke = min(ke, t.m0 + TC_BM);
  kb = (kb / TC_KS) * TC_KS;
  t.kb = kb;
  t.nst = ke > kb ? (ke - kb + TC_KS - 1) / TC_KS : 0;
  return t;
}

template <int S>
__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, TcArgs g) {
  using Cf = TcCfg<S>;
  constexpr int TC_NSTAGE = Cf::NSTAGE, TC_STAGE = Cf::STAGE, TC_A_STAGE = Cf::A_STAGE;
  constexpr int TC_NACC = Cf::NACC, TC_NEXACT = Cf::NEXACT;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full_bar[TC_NSTAGE_MAX], empty_bar[TC_NSTAGE_MAX];
  __shared__ __align__(8) uint64_t accf_bar, acce_bar, done_bar, probe_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  volatile int* abort_v = &abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tiles = (g.mpad / TC_BM) * g.tiles_n * g.batch * g.ksplit;

  if (tid == 0) {
    for (int i = 0; i < TC_NSTAGE; ++i) {
      mbar_init(smem_u32(&full_bar[i]), 1);
      mbar_init(smem_u32(&empty_bar[i]), 1);
    }
    mbar_init(smem_u32(&accf_bar), 1);
    mbar_init(smem_u32(&acce_bar), 32 * TC_EPI_WARPS);
    mbar_init(smem_u32(&done_bar), 1);
    mbar_init(smem_u32(&probe_bar), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(TC_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  auto fail = [&]() {
    *abort_v = 1;
    atomicExch(g.err, 1);
  };

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      if (g.probe_wait > 0 && !mbar_wait(smem_u32(&probe_bar), 0u, abort_v, g.probe_wait)) fail();
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&mapA) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&mapB) : "memory");
      long long j = 0;
      for (int it = blockIdx.x; it < tiles && !*abort_v; it += gridDim.x) {
        const TcItem t = tc_item(g, it);
        if (t.skip) continue;
        const int Q = g.nsum * t.nst;
        for (int q = 0; q < Q && !*abort_v; ++q, ++j) {
          const int slot = (int)(j % TC_NSTAGE), round = (int)(j / TC_NSTAGE);
          if (!mbar_wait(smem_u32(&empty_bar[slot]), (uint32_t)((round & 1) ^ 1), abort_v)) {
            if (!*abort_v) fail();
            break;
          }
          const int js = q / t.nst, k0 = t.kb + (q % t.nst) * TC_KS;
          const int bj = t.b * g.nsum + js;
          const uint32_t dA = smem_u32(smem + slot * TC_STAGE), dB = dA + TC_A_STAGE;
          const uint32_t fb = smem_u32(&full_bar[slot]);
          mbar_expect_tx(fb, TC_STAGE);
          tma_load5(dA, &mapA, 0, t.m0, 0, k0 / 8, bj, fb);
          tma_load5(dB, &mapB, 0, t.n0, 0, k0 / 8, bj, fb);
        }
      }
      // no copy may still be writing shared memory when the CTA exits: the
      // last TC_NSTAGE stages issued (one per slot) must have landed
      for (long long jj = j > TC_NSTAGE ? j - TC_NSTAGE : 0; jj < j; ++jj)
        if (!mbar_wait(smem_u32(&full_bar[jj % TC_NSTAGE]), (uint32_t)((jj / TC_NSTAGE) & 1), nullptr)) fail();
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      long long j = 0;
      unsigned cycle = 0;
      const uint32_t a_base = smem_u32(smem);
      for (int it = blockIdx.x; it < tiles && !*abort_v; it += gridDim.x) {
        const TcItem t = tc_item(g, it);
        if (t.skip) continue;
        const int Q = g.nsum * t.nst;
        const int nchunks = Q > 0 ? ceil_div_d(Q, TC_DRAIN_STAGES) : 1;
        bool ok = true;
        for (int c = 0; c < nchunks && ok; ++c) {
          // accumulators drained and zeroed by the epilogue
          if (!mbar_wait(smem_u32(&acce_bar), cycle & 1u, abort_v)) {
            if (!*abort_v) fail();
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const int q1 = min(Q, (c + 1) * TC_DRAIN_STAGES);
          for (int q = c * TC_DRAIN_STAGES; q < q1; ++q, ++j) {
            const int slot = (int)(j % TC_NSTAGE), round = (int)(j / TC_NSTAGE);
            if (!mbar_wait(smem_u32(&full_bar[slot]), (uint32_t)(round & 1), abort_v)) {
              if (!*abort_v) fail();
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t sa = a_base + slot * TC_STAGE, sb = sa + TC_A_STAGE;
#pragma unroll
            for (int s1 = 1; s1 <= S; ++s1) {
              const int ntot = TC_BN * (S + 1 - s1);
#pragma unroll
              for (int c0 = 0; c0 < ntot; c0 += 256) {
                const int nn = min(256, ntot - c0);
                const uint64_t ad = smem_desc(sa + (s1 - 1) * TC_BM * 16, Cf::LBO_A, 128);
                const uint64_t bd = smem_desc(sb + c0 * 16, Cf::LBO_B, 128);
                mma_bf16(tmem + (uint32_t)(TC_BN * (s1 - 1) + c0), ad, bd, idesc_bf16(TC_BM, nn));
              }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&empty_bar[slot])));
          }
          if (!ok) break;
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&accf_bar)));
          ++cycle;
        }
        if (!ok) break;
      }
      // every MMA issued has completed before TMEM is released
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&done_bar)));
      if (!mbar_wait(smem_u32(&done_bar), 0u, nullptr)) fail();
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int lq = warp & 3, ch = (warp - 2) >> 2;  // TMEM lane quarter, column quarter
    const uint32_t tmem_row = tmem + ((uint32_t)(32 * lq) << 16) + (uint32_t)(TC_CPT * ch);
    const bool aunit = g.alpha == 1.0 || g.alpha == -1.0;
    const unsigned long long asgn = (aunit && g.alpha < 0.0) ? (1ull << 63) : 0ull;
    const uint32_t acce = smem_u32(&acce_bar), accf = smem_u32(&accf_bar);
    // zero every accumulator, then hand them to the MMA issuer
#pragma unroll
    for (int a = 0; a < TC_NACC; ++a) tmem_zero16(tmem_row + (uint32_t)(a * TC_BN));
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    mbar_arrive(acce);
    unsigned cycle = 0;
    for (int it = blockIdx.x; it < tiles; it += gridDim.x) {
      const TcItem t = tc_item(g, it);
      if (t.skip) continue;
      const int row = t.m0 + 32 * lq + lane;
      const int cbase = t.n0 + TC_CPT * ch;
      const int ea = row < g.m ? g.ea[(long long)t.b * g.mpad + row] : 0;
      const int z = t.b * g.ksplit + t.kpart;
      double* C = g.C + (long long)z * g.sC * g.es;
      const double* Cin =
          (g.Cin && t.kpart == 0 && g.beta != 0.0) ? g.Cin + (long long)(t.b / g.bdivC) * g.sCin * g.es : nullptr;
      const int Q = g.nsum * t.nst;
      const int nchunks = Q > 0 ? ceil_div_d(Q, TC_DRAIN_STAGES) : 1;
      long long I[TC_CPT];
#pragma unroll
      for (int jj = 0; jj < TC_CPT; ++jj) I[jj] = 0;
      bool flushed = false;
      int ndrain = 0;
      for (int c = 0; c < nchunks; ++c) {
        // uniform over the warp: the TMEM accesses below are warp-collective
        const bool ok = __all_sync(0xffffffffu, !*abort_v && mbar_wait(accf, cycle & 1u, abort_v));
        if (!ok) {
          if (!*abort_v) fail();
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const bool last = c + 1 == nchunks;
        drain_exact<TC_NEXACT>(tmem_row, I);
#pragma unroll
        for (int a = 0; a < TC_NEXACT; ++a) tmem_zero16(tmem_row + (uint32_t)(a * TC_BN));
        // |I| grows by < 2^56.1 per drain: every max_drains drains the
        // partial sum is written out before it can leave int64 (K > ~15k)
        const bool flush = !last && ++ndrain == g.max_drains;
        // acc7 + acc8 (only at the end) into registers, then the TMEM goes
        // back to the MMA issuer: the next tile's MMAs run while this thread
        // builds and writes its FP64 outputs
        float a7[TC_CPT];
#pragma unroll
        for (int jj = 0; jj < TC_CPT; ++jj) a7[jj] = 0.0f;
        if (last && S >= 6) {
#pragma unroll
          for (int h = 0; h < TC_CPT; h += 8) {
            uint32_t r7[8], r8[8];
#pragma unroll
            for (int j2 = 0; j2 < 8; ++j2) r8[j2] = 0u;
            tmem_ld8(tmem_row + (uint32_t)(5 * TC_BN + h), r7);
            if (S >= 7) tmem_ld8(tmem_row + (uint32_t)(6 * TC_BN + h), r8);
#pragma unroll
            for (int j2 = 0; j2 < 8; ++j2) a7[h + j2] = __uint_as_float(r7[j2]) + __uint_as_float(r8[j2]);
          }
#pragma unroll
          for (int a = TC_NEXACT; a < TC_NACC; ++a) tmem_zero16(tmem_row + (uint32_t)(a * TC_BN));
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        mbar_arrive(acce);
        ++cycle;
        if ((last || flush) && row < g.m) {
          // value = (I + 2^32 (acc7 + acc8)) 2^(ea + eb - 48), then alpha and beta
#pragma unroll
          for (int jj = 0; jj < TC_CPT; ++jj) {
            const int col = cbase + jj;
            if (col < g.n) {
              // while |I| < 2^55, I 2^8 plus acc7 rounded at 2^-40 stays
              // exact to 2^-57 of the operands' row x column maxima; above,
              // acc7 rounded at 2^-32 is below 2^-56 of the result
              long long J = I[jj];
              int e = ea + g.eb[(long long)t.b * g.npad + col] - 48;
              const bool fine = J > -(1LL << 55) && J < (1LL << 55);
              const float tt = a7[jj] * (fine ? 0x1p40f : 0x1p32f);
              const long long add = fabsf(tt) < 2147483648.0f ? (long long)__float2int_rn(tt) : __float2ll_rn(tt);
              if (fine) {
                J = J * 256 + add;
                e -= 8;
              } else {
                J += add;
              }
              double v = fix_to_double(J, e);
              if (aunit) v = __longlong_as_double(__double_as_longlong(v) ^ (long long)asgn);
              else v *= g.alpha;
              const long long ic = (row + (long long)col * g.ldc) * g.es;
              if (flushed) v += C[ic];
              else if (Cin) v = fma(g.beta, Cin[(row + (long long)col * g.ldcin) * g.es], v);
              C[ic] = v;
            }
          }
        }
        if (flush) {
#pragma unroll
          for (int jj = 0; jj < TC_CPT; ++jj) I[jj] = 0;
          flushed = true;
          ndrain = 0;
        }
      }
      if (*abort_v && row < g.m) {  // unfinished tile: NaN outputs
#pragma unroll
        for (int jj = 0; jj < TC_CPT; ++jj)
          if (cbase + jj < g.n) C[(row + (long long)(cbase + jj) * g.ldc) * g.es] = NAN;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
}

// ---- slicing: exponents of rows of op(A) (cols of op(B)) then the 7 slices

// Slicing works on 64 x 64 tiles of op(X_{b,j}) staged in shared memory, so
// that global reads follow the memory order of X (op N: i fastest, op T: k
// fastest) and the slice writes follow the [i][k] (k fastest) order.
constexpr int SL_T = 64;

// Per-term weights w_j of a grouped sum, passed by value (no host-to-device
// copy, so the whole product can be captured in a CUDA graph).
struct TermWeights {
  double w[MAX_SUM];
};

__device__ __forceinline__ void load_tile(double (*tile)[SL_T + 1], const double* X, int ld, int op, int rows, int K,
                                          int i0, int k0, double wj, const int* ek, int sgn, int es) {
  for (int e = threadIdx.x; e < SL_T * SL_T; e += blockDim.x) {
    // a = fastest index in memory, c = the other
    const int a = e % SL_T, c = e / SL_T;
    int i, k;
    if (op == OP_N) { i = i0 + a; k = k0 + c; }
    else { k = k0 + a; i = i0 + c; }
    double v = 0.0;
    if (i < rows && k < K) {
      v = wj * (op == OP_N ? X[es * (i + (long long)k * ld)] : X[es * (k + (long long)i * ld)]);
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
                                  long long sXj, int bdiv, TermWeights w, int rpad, int* e, const int* ek,
                                  int ekpad, int sgn, int es) {
  __shared__ double tile[SL_T][SL_T + 1];
  const int i0 = blockIdx.x * SL_T, k0 = blockIdx.y * SL_T;
  const int b = blockIdx.z / nsum, js = blockIdx.z % nsum;
  load_tile(tile, X + (long long)(b / bdiv) * sX * es + js * sXj, ld, op, rows, K, i0, k0, w.w[js],
            ek ? ek + (long long)b * ekpad : nullptr, sgn, es);
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

// slices q~_s (s = 1..7) of w_j op(X_{b,j}) 2^-e_i, stored as
// [b][j][k / 8][s][i][k % 8] (rpad rows, kpad / 8 groups of 8 k): the
// layout the kernel's 5-D TMA boxes read as K-major core matrices
template <int S>
__global__ void tc_slice_kernel(int rows, int K, int nsum, int op, const double* X, int ld, long long sX, long long sXj,
                                int bdiv, TermWeights w, const int* e, int rpad, int kpad, __nv_bfloat16* out,
                                long long sOut, const int* ek, int sgn, int es) {
  __shared__ double tile[SL_T][SL_T + 1];
  const int i0 = blockIdx.x * SL_T, k0 = blockIdx.y * SL_T;
  const int b = blockIdx.z / nsum, js = blockIdx.z % nsum;
  load_tile(tile, X + (long long)(b / bdiv) * sX * es + js * sXj, ld, op, rows, K, i0, k0, w.w[js],
            ek ? ek + (long long)b * kpad : nullptr, sgn, es);
  __syncthreads();
  __nv_bfloat16* o = out + ((long long)b * nsum + js) * sOut;
  const long long sl_stride = (long long)rpad * 8;  // next slice within a k group
  for (int t = threadIdx.x; t < SL_T * SL_T; t += blockDim.x) {
    // 8 consecutive k of 4 consecutive rows per warp: 64 contiguous bytes per slice
    const int k8 = t & 7, ii = (t >> 3) & (SL_T - 1), kg = t >> 9;
    const int kk = kg * 8 + k8;
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
      const int sh = 8 * S - ei;  // in [-968, 1130] for finite nonzero data
      // 2^sh as two exact, normal powers of two
      const int s1 = sh / 2, s2 = sh - s1;
      X = __double2ll_rn(v * __longlong_as_double((long long)(1023 + s1) << 52) *
                         __longlong_as_double((long long)(1023 + s2) << 52));
    }
    int q[S];
#pragma unroll
    for (int sidx = S - 1; sidx >= 1; --sidx) {
      const int d = (int)((X + 128) & 255) - 128;
      q[sidx] = d;
      X = (X - d) >> 8;
    }
    q[0] = (int)X;
    __nv_bfloat16* dst = o + ((long long)(k >> 3) * S * rpad + i) * 8 + (k & 7);
#pragma unroll
    for (int sidx = 0; sidx < S; ++sidx)
      dst[sidx * sl_stride] = __float2bfloat16_rn((float)q[sidx] * __int_as_float((127 - 8 * sidx) << 23));
  }
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
// (no link-time dependence on the driver library)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    else
      cudaGetLastError();
  });
  return fn;
}

// 5-D map over a slice set [nbj][kpad / 8][7][rpad][8] (BF16): box = 8 k x
// box_rows rows x 7 slices x 2 k groups (one 16-wide stage) x 1 term
void make_slice_map(CUtensorMap* map, const __nv_bfloat16* base, int rpad, int kpad, int nbj, int box_rows, int S) {
  auto enc = tensor_map_encoder();
  if (!enc) throw CudaFail{cudaErrorNotSupported, __FILE__, __LINE__};
  const cuuint64_t dims[5] = {8, (cuuint64_t)rpad, (cuuint64_t)S, (cuuint64_t)(kpad / 8), (cuuint64_t)nbj};
  const cuuint64_t strides[4] = {16, (cuuint64_t)16 * rpad, (cuuint64_t)16 * rpad * S,
                                 (cuuint64_t)16 * rpad * S * (kpad / 8)};
  const cuuint32_t box[5] = {8, (cuuint32_t)box_rows, (cuuint32_t)S, TC_KS / 8, 1};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, (void*)base, dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw CudaFail{cudaErrorInvalidValue, __FILE__, __LINE__};
}

int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
  }
  return sms;
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
  // The tile is 128 x 64 with a 16-wide k stage.  Full tiles: m >= 128,
  // n >= 64, k >= 64.  A short side still pays when K is long: a product
  // with m or n down to 32 fills a quarter / half of each tile, but GB300's
  // FP64 pipe is ~20x slower than the sliced tensor-core rate, so products
  // with k >= 512 (the W = Y^* C panels of the blocked QR) also go there.
  if (!(t_tc.enabled && t_tc.ar && ((t_tc.sites >> g.site) & 1u) && tc_gemm_supported(g))) return false;
  if (g.m >= TC_BM && g.n >= TC_BN && g.k >= 64) return true;
  return g.m >= 32 && g.n >= 32 && g.k >= 512;
}

template <int S>
void tc_gemm_s(const GemmArgs<double>& g, cudaStream_t st, Arena& ar, int* err) {
  using Cf = TcCfg<S>;
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
  const long long sAsl = (long long)S * mpad * kpad, sBsl = same ? sAsl : (long long)S * npad * kpad;
  __nv_bfloat16* Asl = ar.get<__nv_bfloat16>((size_t)sAsl * nsum * g.batch);
  __nv_bfloat16* Bsl = same ? Asl : ar.get<__nv_bfloat16>((size_t)sBsl * nsum * g.batch);
  int* ea = ar.get<int>((size_t)mpad * g.batch);
  int* eb = same ? ea : ar.get<int>((size_t)npad * g.batch);
  // term weights apply to A; B gets unit weights
  TermWeights w, wunit;
  for (int j = 0; j < MAX_SUM; ++j) { w.w[j] = g.w[j]; wunit.w[j] = 1.0; }
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
                                          wunit, kpad, ek, nullptr, 0, 0, g.es);
    ZCSD_LAUNCH();
  }
  tc_row_exp_kernel<<<ga, 256, 0, st>>>(g.m, g.k, nsum, opA, g.A, g.lda, g.sA, g.sAj, g.bdivA, w, mpad, ea, ek, kpad,
                                        1, g.es);
  ZCSD_LAUNCH();
  if (!same) {
    tc_row_exp_kernel<<<gb, 256, 0, st>>>(g.n, g.k, nsum, opBt, g.B, g.ldb, g.sB, g.sBj, g.bdivB, wunit, npad,
                                          eb, ek, kpad, -1, g.es);
    ZCSD_LAUNCH();
  }
  tc_slice_kernel<S><<<ga, 256, 0, st>>>(g.m, g.k, nsum, opA, g.A, g.lda, g.sA, g.sAj, g.bdivA, w, ea, mpad, kpad, Asl,
                                      sAsl, ek, 1, g.es);
  ZCSD_LAUNCH();
  if (!same) {
    tc_slice_kernel<S><<<gb, 256, 0, st>>>(g.n, g.k, nsum, opBt, g.B, g.ldb, g.sB, g.sBj, g.bdivB, wunit, eb, npad,
                                        kpad, Bsl, sBsl, ek, -1, g.es);
    ZCSD_LAUNCH();
  }
  TcArgs t;
  t.m = g.m; t.n = g.n; t.kpad = kpad; t.nsum = nsum; t.batch = g.batch;
  t.ea = ea; t.eb = eb; t.mpad = mpad;
  t.npad = same ? mpad : npad;  // row pitch of the B slices and exponents
  t.tiles_n = npad / TC_BN;
  t.kb_flags = g.kflags; t.ksplit = std::max(1, g.ksplit); t.uplo = g.uplo; t.alpha = re(g.alpha); t.beta = re(g.beta);
  t.Cin = g.Cin; t.ldcin = g.ldcin; t.sCin = g.sCin; t.bdivC = g.bdivC;
  t.C = g.C; t.ldc = g.ldc; t.sC = g.sC; t.err = err;
  t.es = g.es;
  t.max_drains = t_tc.flush_every > 0 ? std::min(t_tc.flush_every, TC_MAX_DRAINS) : TC_MAX_DRAINS;
  t.probe_wait = t_tc.probe_wait;
  CUtensorMap mapA, mapB;
  make_slice_map(&mapA, Asl, mpad, kpad, g.batch * nsum, TC_BM, S);
  make_slice_map(&mapB, Bsl, t.npad, kpad, g.batch * nsum, TC_BN, S);
  static std::once_flag attr_once;
  std::call_once(attr_once, [] {
    cudaFuncSetAttribute(tc_gemm_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cf::SMEM);
  });
  const long long items = (long long)(mpad / TC_BM) * (npad / TC_BN) * g.batch * t.ksplit;
  const int grid = (int)std::min<long long>(items, num_sms());
  tc_gemm_kernel<S><<<grid, TC_THREADS, Cf::SMEM, st>>>(mapA, mapB, t);
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


bool tc_will_handle_complex(const GemmArgs<z64>& g) {
  // one complex product = two real grouped sums over the interleaved parts;
  // grouped complex sums and the inner-dimension-balanced product stay on
  // the FP64 pipe, as do complex alpha / beta
  if (g.nsum != 1 || g.kbal || g.alpha.y != 0.0 || g.beta.y != 0.0) return false;
  GemmArgs<double> r;
  r.m = g.m; r.n = g.n; r.k = g.k; r.site = g.site; r.ksplit = std::max(1, g.ksplit);
  return tc_will_handle(r);
}

void tc_gemm_complex(const GemmArgs<z64>& g, cudaStream_t st, Arena& ar, int* err) {
  // op(A) = A, A^T or A^*: Re op(A) = op'(Re A), Im op(A) = sA op'(Im A)
  // with op' the real N / T and sA = -1 for the conjugate transpose
  const double sa = g.opA == OP_C ? -1.0 : 1.0, sb = g.opB == OP_C ? -1.0 : 1.0;
  GemmArgs<double> r;
  r.m = g.m; r.n = g.n; r.k = g.k;
  r.opA = g.opA == OP_N ? OP_N : OP_T;
  r.opB = g.opB == OP_N ? OP_N : OP_T;
  r.lda = g.lda; r.sA = g.sA; r.ldb = g.ldb; r.sB = g.sB;
  r.ldcin = g.ldcin; r.sCin = g.sCin; r.ldc = g.ldc; r.sC = g.sC;
  r.batch = g.batch; r.bdivA = g.bdivA; r.bdivB = g.bdivB; r.bdivC = g.bdivC;
  r.uplo = g.uplo; r.kflags = g.kflags; r.site = g.site; r.ksplit = g.ksplit;
  r.alpha = g.alpha.x; r.beta = g.beta.x;
  r.nsum = 2;
  r.es = 2;
  const double* A = reinterpret_cast<const double*>(g.A);
  const double* B = reinterpret_cast<const double*>(g.B);
  const double* Ci = reinterpret_cast<const double*>(g.Cin);
  double* C = reinterpret_cast<double*>(g.C);
  // Re C = Re op(A) Re op(B) - Im op(A) Im op(B)
  GemmArgs<double> re_ = r;
  re_.A = A; re_.sAj = 1;
  re_.B = B; re_.sBj = 1;
  re_.w[0] = 1.0; re_.w[1] = -sa * sb;
  re_.Cin = Ci; re_.C = C;
  tc_gemm(re_, st, ar, err);
  // Im C = Re op(A) Im op(B) + Im op(A) Re op(B)
  GemmArgs<double> im_ = r;
  im_.A = A; im_.sAj = 1;
  im_.B = B + 1; im_.sBj = -1;
  im_.w[0] = sb; im_.w[1] = sa;
  im_.Cin = Ci ? Ci + 1 : nullptr; im_.C = C + 1;
  tc_gemm(im_, st, ar, err);
}

void tc_gemm(const GemmArgs<double>& g, cudaStream_t st, Arena& ar, int* err) {
  // fewer slices (40 or 48 bits) only for the call sites the caller marked
  // as well conditioned; everything else keeps 7 (FP64-accurate)
  const int S = ((t_tc.reduced_sites >> g.site) & 1u) ? t_tc.reduced_slices : TC_SMAX;
  if (S == 5) tc_gemm_s<5>(g, st, ar, err);
  else if (S == 6) tc_gemm_s<6>(g, st, ar, err);
  else tc_gemm_s<7>(g, st, ar, err);
}

}  // namespace zcsd
