// Zolo-eig (Section 5): eigendecomposition of a Hermitian matrix by spectral
// divide and conquer on the polar factor of a shifted block.
//
// A split of block B_sub (sz x sz) at the shift s: W = polar((B_sub - sI) /
// ||B_sub - sI||_F) by Zolo-pd, P = (W + I)/2 projects onto the eigenvectors
// above s, k = trace(P) of them; [Q1 Q2] = qr(P Omega) with Omega Gaussian
// gives Q1 spanning range(P), and Q^* B_sub Q is block diagonal up to
// ||B'_21||_F, which is the backward error of the split.
//
// The recursion runs level by level.  Every block of a level that still
// needs a split goes through the same launches: the blocks form groups
// (chosen by a cost model), each block is padded to the group's largest
// size nb with an identity block, X_p = diag((B_p - s_p I) / ||B_p - s_p I||_F, I), and one
// batched Zolo-pd, one batched QR and batched products serve the whole
// group.  The padding is exactly decoupled: polar(diag(X, I)) = diag(polar(X),
// I); with P padded by zeros, P Omega has zero rows below sz_p, so every
// Householder reflector is zero there and Q = diag(Q_p, I) exactly.  The
// host reads the per-block scalars (norms, medians, traces, off-block
// norms) once per level and attempt, not once per block.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "solver.h"

namespace zcsd {

namespace {

__device__ inline double eig_block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
  __syncthreads();
  return r;
}

// Problem p of a batched reduction: the m_p x c_p block at X + boff_p
// (leading dimension ld), shift_p subtracted on its diagonal (shift may be
// null: no shift).
struct RedTab {
  const long long* boff;
  const int* m;
  const int* c;
  const double* shift;
};

constexpr int RED_PARTS = 32;  // partial sums per problem (fixed order: deterministic)

template <class T>
__global__ void blk_fro2_partial(const T* X, int ld, RedTab t, double* part) {
  __shared__ double sh[32];
  const int p = blockIdx.y, m = t.m[p], c = t.c[p];
  const double s = t.shift ? t.shift[p] : 0.0;
  const T* Xp = X + t.boff[p];
  const long long total = (long long)m * c;
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % m), j = (int)(e / m);
    T x = Xp[i + (long long)j * ld];
    if (i == j) x = sub(x, from_re<T>(s));
    acc += abs2(x);
  }
  const double r = eig_block_sum(acc, sh);
  if (threadIdx.x == 0) part[(long long)p * gridDim.x + blockIdx.x] = r;
}

__global__ void blk_finish(const double* part, int nparts, double* out) {
  __shared__ double sh[32];
  const int p = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += part[(long long)p * nparts + i];
  const double r = eig_block_sum(acc, sh);
  if (threadIdx.x == 0) out[p] = r;
}

// d[off_p + i] = Re B[off_p + i, off_p + i]
template <class T>
__global__ void blk_diag(const T* B, int n, const int* off, const int* sz, double* d) {
  const int p = blockIdx.y, o = off[p];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < sz[p]; i += gridDim.x * blockDim.x)
    d[o + i] = re(B[(long long)(o + i) * (n + 1)]);
}

// out[p] = lower median of d[off_p .. off_p + sz_p) (rank counting, one CTA)
__global__ void blk_median(const double* d, const int* off, const int* sz, double* out) {
  const int p = blockIdx.x, m = sz[p];
  const double* dp = d + off[p];
  const int want = (m - 1) / 2;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double v = dp[i];
    int less = 0, eq_before = 0;
    for (int k = 0; k < m; ++k) {
      const double w = dp[k];
      less += (w < v);
      eq_before += (w == v && k < i);
    }
    if (less + eq_before == want) out[p] = v;
  }
}

// X_p = diag((B_p - s_p I) / xn_p, I), nb x nb, B_p the sz_p block at (off_p, off_p)
template <class T>
__global__ void blk_gather_pad(const T* B, int n, const int* off, const int* sz, const double* s,
                               const double* xn, int nb, T* X) {
  const int p = blockIdx.y, o = off[p], m = sz[p];
  const double sp = s[p], inv = 1.0 / xn[p];
  const long long nn = (long long)nb * nb;
  T* Xp = X + p * nn;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % nb), j = (int)(e / nb);
    T v;
    if (i < m && j < m) {
      v = B[(o + i) + (long long)(o + j) * n];
      if (i == j) v = sub(v, from_re<T>(sp));
      v = scal(inv, v);
    } else {
      v = from_re<T>(i == j ? 1.0 : 0.0);
    }
    Xp[e] = v;
  }
}

// tr_p = sum_{j < sz_p} (Re W_p[j, j] + 1) / 2 = trace of P_p
template <class T>
__global__ void blk_trace_half(const T* W, int nb, const int* sz, double* out) {
  __shared__ double sh[32];
  const int p = blockIdx.x, m = sz[p];
  const T* Wp = W + (long long)p * nb * nb;
  double acc = 0.0;
  for (int j = threadIdx.x; j < m; j += blockDim.x) acc += 0.5 * (re(Wp[j + (long long)j * nb]) + 1.0);
  const double r = eig_block_sum(acc, sh);
  if (threadIdx.x == 0) out[p] = r;
}

// P_p = (W_p + I) / 2 on the leading sz_p x sz_p block, zero elsewhere
template <class T>
__global__ void blk_proj_pad(const T* W, int nb, const int* sz, T* Pm) {
  const int p = blockIdx.y, m = sz[p];
  const long long nn = (long long)nb * nb;
  const T* Wp = W + p * nn;
  T* Pp = Pm + p * nn;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % nb), j = (int)(e / nb);
    T v = zero<T>();
    if (i < m && j < m) {
      v = scal(0.5, Wp[e]);
      if (i == j) v = add(v, from_re<T>(0.5));
    }
    Pp[e] = v;
  }
}

// accepted problems: B block (off_p, off_p) <- xn_p Om_p[:sz_p, :sz_p] + s_p I
template <class T>
__global__ void blk_writeback(const T* Om, int nb, const int* off, const int* sz, const double* s, const double* xn,
                              const int* accept, T* B, int n) {
  const int p = blockIdx.y;
  if (!accept[p]) return;
  const int o = off[p], m = sz[p];
  const double sp = s[p], a = xn[p];
  const T* Op = Om + (long long)p * nb * nb;
  const long long mm = (long long)m * m;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < mm;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % m), j = (int)(e / m);
    T v = scal(a, Op[i + (long long)j * nb]);
    if (i == j) v = add(v, from_re<T>(sp));
    B[(o + i) + (long long)(o + j) * n] = v;
  }
}

int ew_grid(long long per_problem) { return (int)std::min<long long>((per_problem + 255) / 256, 128); }

// Device copy of a small host table (pageable source: the call returns once
// the data is staged, so the host vector may go out of scope afterwards).
template <class X>
X* upload(Arena& ar, cudaStream_t st, const std::vector<X>& h) {
  X* d = ar.get<X>(std::max<size_t>(h.size(), 1));
  if (!h.empty()) ZCSD_CUDA(cudaMemcpyAsync(d, h.data(), sizeof(X) * h.size(), cudaMemcpyHostToDevice, st));
  return d;
}

template <class X>
std::vector<X> download(Ctx& cx, const X* d, size_t count) {
  std::vector<X> h(count);
  if (count) d2h(cx, h.data(), d, sizeof(X) * count);
  return h;
}

// ||X_p - shift_p I||_F^2 of every problem of a reduction table (device out)
template <class T>
void blk_fro2(cudaStream_t st, Arena& ar, const T* X, int ld, const std::vector<long long>& boff,
              const std::vector<int>& m, const std::vector<int>& c, const double* dshift, double* out) {
  const int P = (int)boff.size();
  if (P == 0) return;
  RedTab t;
  t.boff = upload(ar, st, boff);
  t.m = upload(ar, st, m);
  t.c = upload(ar, st, c);
  t.shift = dshift;
  double* part = ar.get<double>((size_t)P * RED_PARTS);
  blk_fro2_partial<T><<<dim3(RED_PARTS, P), 256, 0, st>>>(X, ld, t, part);
  ZCSD_LAUNCH();
  blk_finish<<<P, 256, 0, st>>>(part, RED_PARTS, out);
  ZCSD_LAUNCH();
}

struct EigBlk {
  int off, sz;
  bool top;
};

// Per-block state of a level across its split attempts.
struct SplitState {
  EigBlk b;
  double s0 = 0.0, spread = 0.0, s = 0.0, xn = 0.0, scal_tol = 0.0, off_tol = 0.0;
  bool done = false;
};

}  // namespace

// Eigendecomposition of the Hermitian n x n matrix Bin (device, ld ldb) by
// spectral divide and conquer (Section 5).  Writes lam (device, length n) and
// V (device, ld n).  If split_at is finite, only eigenpairs below it are
// computed (Section 5.2: split at 1.1 for Algorithm 3); they occupy columns
// [*lo, n) on return.  Eigenvalues in [*lo, n) are sorted ascending with V.
template <class T>
void heig_impl(Ctx& cx, Arena& ar, int n, const T* Bin, int ldb, double* lam, T* V, double split_at, int* lo_out,
               EigDiag* ed) {
  cudaStream_t st = cx.stream;
  const long long nn = (long long)n * n;
  const size_t mk = ar.mark();
  T* Bw = ar.get<T>(nn);
  T* Vt = ar.get<T>(nn);  // n x sz scratch of the eigenvector updates
  double* dvals = ar.get<double>(n);
  double* lamw = ar.get<double>(n);
  double* sc = ar.get<double>(64);
  double* scratch = ar.get<double>(304 * 4);
  int* perm = ar.get<int>(n);
  symmetrize<T>(st, n, Bin, ldb, 0, Bw, n, 0, 1);
  set_eye<T>(st, n, n, V, n, 0, 1);
  fro2<T>(st, n, n, Bw, n, 0, 0.0, sc, 1, scratch);
  const double bnorm = std::sqrt(download(cx, sc, 1)[0]);
  static const bool debug = getenv("ZCSD_DEBUG") != nullptr;
  const bool restricted = std::isfinite(split_at);
  const T one = from_re<T>(1.0), zer = zero<T>();

  std::vector<EigBlk> level{{0, n, true}};
  std::vector<int> leaf_off, leaf_sz;  // negative size: a scalar block (keeps its diagonal)
  int lo = 0;
  for (int depth = 0; !level.empty(); ++depth) {
    std::vector<SplitState> work;
    for (const EigBlk& b : level) {
      if (b.sz <= 0) continue;
      if (b.sz <= cx.eig_leaf && !(b.top && restricted)) {
        leaf_off.push_back(b.off);
        leaf_sz.push_back(b.sz);
      } else {
        SplitState s;
        s.b = b;
        work.push_back(s);
      }
    }
    level.clear();
    if (work.empty()) break;
    const size_t mlev = ar.mark();
    const int P = (int)work.size();
    // ---- the median of diag(B_p) (the first shift), all blocks of the level
    {
      std::vector<int> off(P), sz(P);
      for (int p = 0; p < P; ++p) {
        off[p] = work[p].b.off;
        sz[p] = work[p].b.sz;
      }
      double* d = ar.get<double>(P);
      const int* doff = upload(ar, st, off);
      const int* dsz = upload(ar, st, sz);
      blk_diag<T><<<dim3(8, P), 256, 0, st>>>(Bw, n, doff, dsz, dvals);
      ZCSD_LAUNCH();
      blk_median<<<P, 256, 0, st>>>(dvals, doff, dsz, d);
      ZCSD_LAUNCH();
      const std::vector<double> h = download(cx, d, P);
      for (int p = 0; p < P; ++p) {
        SplitState& w = work[p];
        const double sz_d = (double)w.b.sz;
        w.s0 = (w.b.top && restricted) ? split_at : h[p];
        // Accepted rounding levels, against ||B||_F of the whole matrix (the
        // backward error of the eigendecomposition is relative to it): a
        // block within scal_tol of s I is scalar; a split is accepted when
        // ||B'_21||_F <= off_tol.  With at most ~log2(n / 64) levels of
        // splits, 2 n u ||B||_F per split keeps the eigendecomposition's
        // share of the CSD backward error (Theorem 3.1, term Delta B_2) near
        // 12 n u, inside the 50 n u bound; small blocks keep 50 sqrt(sz) u.
        w.scal_tol = 100.0 * U_ROUND * bnorm * std::sqrt(sz_d);
        w.off_tol = std::max(50.0 * std::sqrt(sz_d), 2.0 * n) * U_ROUND * bnorm;
      }
    }
    for (int attempt = 0; attempt < 7; ++attempt) {
      std::vector<int> pend;
      for (int p = 0; p < P; ++p)
        if (!work[p].done) pend.push_back(p);
      if (pend.empty()) break;
      const size_t matt = ar.mark();
      const int Q = (int)pend.size();
      if (attempt > 0) ed->retries += Q;
      // ---- shifts: the median, then s0 + (+1, -1, +2, -2, +4, -4) * 0.05 *
      // spread, inside the block's spectrum (which may be a cluster much
      // narrower than ||B_sub||)
      std::vector<double> shift(Q);
      for (int q = 0; q < Q; ++q) {
        SplitState& w = work[pend[q]];
        if (attempt == 0) {
          w.s = w.s0;
        } else {
          const double mag = (double)(1 << ((attempt - 1) / 2)) * (attempt & 1 ? 1.0 : -1.0);
          w.s = w.s0 + 0.05 * mag * w.spread;
        }
        shift[q] = w.s;
      }
      // ---- ||B_p - s_p I||_F
      std::vector<int> act;
      {
        std::vector<long long> boff(Q);
        std::vector<int> sz(Q);
        for (int q = 0; q < Q; ++q) {
          boff[q] = (long long)work[pend[q]].b.off * (n + 1);
          sz[q] = work[pend[q]].b.sz;
        }
        const double* dshift = upload(ar, st, shift);
        double* d = ar.get<double>(Q);
        blk_fro2<T>(st, ar, Bw, n, boff, sz, sz, dshift, d);
        const std::vector<double> h = download(cx, d, Q);
        for (int q = 0; q < Q; ++q) {
          SplitState& w = work[pend[q]];
          w.xn = std::sqrt(h[q]);
          if (attempt == 0) w.spread = w.xn / std::sqrt((double)w.b.sz);
          if (w.xn <= w.scal_tol) {
            // B_sub = sI to working precision: every vector is an eigenvector
            if (w.b.top && restricted) lo = (w.s < split_at) ? w.b.off : w.b.off + w.b.sz;
            else { leaf_off.push_back(w.b.off); leaf_sz.push_back(-w.b.sz); }
            w.done = true;
            continue;
          }
          act.push_back(pend[q]);
        }
      }
      // ---- groups: the blocks sorted by size (largest first) cut into
      // contiguous runs, each padded to its largest size nb.  A group's time
      // is modelled as a latency term growing with nb (the sequential panel
      // and Cholesky steps) plus work per padded problem, t = a nb + c Pa
      // nb^3 (a = 0.065 ms, c = 9e-9 ms for real data, fitted to measured
      // group times on GB300); the cuts minimise the modelled total.
      std::sort(act.begin(), act.end(), [&](int a, int b) {
        return work[a].b.sz != work[b].b.sz ? work[a].b.sz > work[b].b.sz : work[a].b.off < work[b].b.off;
      });
      const size_t na = act.size();
      std::vector<size_t> cut(na + 1, 0);
      {
        const double ca = 0.065, cc = 9e-9 * (sizeof(T) == sizeof(double) ? 1.0 : 4.0);
        std::vector<double> best(na + 1, 0.0);  // best[i]: blocks [i, na)
        for (size_t i = na; i-- > 0;) {
          const double nb = work[act[i]].b.sz;
          best[i] = 1e300;
          for (size_t j = i + 1; j <= na; ++j) {
            const double t = ca * nb + cc * (double)(j - i) * nb * nb * nb + best[j];
            if (t < best[i]) {
              best[i] = t;
              cut[i] = j;
            }
          }
        }
      }
      for (size_t g0 = 0, gi = 0; g0 < na; ++gi) {
        const int nb = work[act[g0]].b.sz;
        const size_t g1 = cut[g0];
        const std::vector<int> grp(act.begin() + g0, act.begin() + g1);
        g0 = g1;
        const int Pa = (int)grp.size();
        const long long nbb = (long long)nb * nb;
        const size_t mg = ar.mark();
        if (debug) ZCSD_CUDA(cudaStreamSynchronize(st));
        const auto tg0 = std::chrono::steady_clock::now();
        std::vector<int> off(Pa), sz(Pa);
        std::vector<double> s(Pa), xn(Pa);
        for (int a = 0; a < Pa; ++a) {
          const SplitState& w = work[grp[a]];
          off[a] = w.b.off;
          sz[a] = w.b.sz;
          s[a] = w.s;
          xn[a] = w.xn;
        }
        const int* doff = upload(ar, st, off);
        const int* dsz = upload(ar, st, sz);
        const double* ds = upload(ar, st, s);
        const double* dxn = upload(ar, st, xn);
        T* X = ar.get<T>(nbb * Pa);
        T* Wm = ar.get<T>(nbb * Pa);
        T* Qf = ar.get<T>(nbb * Pa);
        T* Tm = ar.get<T>(nbb * Pa);
        T* Om = ar.get<T>(nbb * Pa);
        double* dtr = ar.get<double>(Pa);
        blk_gather_pad<T><<<dim3(ew_grid(nbb), Pa), 256, 0, st>>>(Bw, n, doff, dsz, ds, dxn, nb, X);
        ZCSD_LAUNCH();
        zolo_pd<T>(cx, ar, nb, Pa, X, Wm, nullptr, 0, (cx.mixed_scope & 2u) ? cx.mixed_slices : 0);
        // ---- P = (W + I)/2, k = trace(P) = number of eigenvalues above s
        blk_trace_half<T><<<Pa, 256, 0, st>>>(Wm, nb, dsz, dtr);
        ZCSD_LAUNCH();
        const std::vector<double> tr = download(cx, dtr, Pa);
        std::vector<int> k(Pa, -1);
        bool any = false;
        for (int a = 0; a < Pa; ++a) {
          SplitState& w = work[grp[a]];
          const int ka = (int)std::floor(tr[a] + 0.5);
          if (debug)
            fprintf(stderr, "zolo-eig: depth=%d off=%d sz=%d nb=%d attempt=%d s=%.17g |B-sI|=%.3e trace=%.6f\n", depth,
                    w.b.off, w.b.sz, nb, attempt, w.s, w.xn, tr[a]);
          if (!(std::fabs(tr[a] - ka) <= 0.25)) continue;
          if (w.b.top && restricted && (ka == 0 || ka == w.b.sz)) {
            // all eigenvalues above / all below the split point
            lo = (ka == w.b.sz) ? w.b.off + w.b.sz : w.b.off;
            if (ka == 0) level.push_back({w.b.off, w.b.sz, false});
            w.done = true;
            continue;
          }
          if (ka == 0 || ka == w.b.sz) continue;
          k[a] = ka;
          any = true;
        }
        if (!any) {
          ar.release(mg);
          continue;
        }
        // ---- [Q1 Q2] = qr(P Omega), Q1 spans range(P) (Q = diag(Q_p, I)).
        // With a square Gaussian Omega the leading k columns of P Omega have
        // a condition number of order k, and so does the error of Q1; a block
        // whose split fails the off-block test gets one step of subspace
        // iteration, Q <- qr(P Q), whose leading columns P Q1 ~ Q1 are well
        // conditioned, before a new shift (and a new polar factor) is tried.
        T* Pm = ar.get<T>(nbb * Pa);
        blk_proj_pad<T><<<dim3(ew_grid(nbb), Pa), 256, 0, st>>>(Wm, nb, dsz, Pm);
        ZCSD_LAUNCH();
        randn<T>(st, nb, nb * Pa, Om, nb,
                 cx.seed + 7919ull * (unsigned long long)(depth * 4096 + attempt * 256 + (int)gi) + 1ull);
        auto bgemm = [&](int opA, const T* A, const T* Bp, T* C) {
          GemmArgs<T> g;
          g.batch = Pa;
          g.m = nb; g.n = nb; g.k = nb; g.opA = opA; g.opB = OP_N;
          g.A = A; g.lda = nb; g.sA = nbb;
          g.B = Bp; g.ldb = nb; g.sB = nbb;
          g.C = C; g.ldc = nb; g.sC = nbb;
          g.alpha = one; g.beta = zer;
          g.site = GS_EIG;
          gemm(g, st);
        };
        std::vector<int> cand;  // blocks with a valid k still to be tested
        for (int a = 0; a < Pa; ++a)
          if (k[a] >= 0) cand.push_back(a);
        for (int pass = 0; pass < 2 && !cand.empty(); ++pass) {
          bgemm(OP_N, Pm, pass == 0 ? Om : Qf, Wm);  // P Omega, then P Q
          {
            const size_t mq = ar.mark();
            QRStore<T> q = qr_alloc<T>(ar, nb, nb, nb, Pa);
            qr_factor<T>(st, ar, q, Wm, nb, nbb);
            qr_form_q<T>(st, ar, q, Qf, nb, nbb);
            ar.release(mq);
          }
          // ---- B' = Q^* B_sub Q = ||B_sub - sI||_F Q^* X Q + s I: the shift
          // is added back exactly, so the departure of Q from orthogonality
          // is multiplied by the small ||B_sub - sI|| (not by |s|) in the
          // off-diagonal block
          bgemm(OP_N, X, Qf, Tm);
          bgemm(OP_C, Qf, Tm, Om);
          std::vector<long long> boff;
          std::vector<int> rm, rc;
          for (int a : cand) {
            boff.push_back((long long)a * nbb + k[a]);
            rm.push_back(sz[a] - k[a]);
            rc.push_back(k[a]);
          }
          double* doffa = ar.get<double>(cand.size());
          blk_fro2<T>(st, ar, Om, nb, boff, rm, rc, nullptr, doffa);
          const std::vector<double> h = download(cx, doffa, cand.size());
          std::vector<int> accept(Pa, 0), retry;
          bool any_acc = false;
          for (size_t i = 0; i < cand.size(); ++i) {
            const int a = cand[i];
            SplitState& w = work[grp[a]];
            const double offa = w.xn * std::sqrt(h[i]);
            if (debug)
              fprintf(stderr, "zolo-eig:   off=%d pass=%d k=%d ||B21||=%.3e tol=%.3e\n", w.b.off, pass, k[a], offa,
                      w.off_tol);
            if (cx.test_flags & TEST_REJECT_EIG_SPLITS) continue;  // injected failure (tests only)
            if (!(offa <= w.off_tol)) {
              retry.push_back(a);
              continue;
            }
            ed->offblock = std::max(ed->offblock, offa / std::max(bnorm, 1e-300));
            ed->splits += 1;
            accept[a] = 1;
            any_acc = true;
            w.done = true;
            const int ka = k[a];
            if (w.b.top && restricted) {
              lo = w.b.off + ka;
              level.push_back({w.b.off + ka, w.b.sz - ka, false});
            } else {
              level.push_back({w.b.off, ka, false});
              level.push_back({w.b.off + ka, w.b.sz - ka, false});
            }
          }
          if (any_acc) {
            // accept: B_sub <- B' (+ s I), V[:, off:off+sz] <- V[:, off:off+sz] Q_p
            const int* dacc = upload(ar, st, accept);
            blk_writeback<T><<<dim3(ew_grid(nbb), Pa), 256, 0, st>>>(Om, nb, doff, dsz, ds, dxn, dacc, Bw, n);
            ZCSD_LAUNCH();
            for (int a = 0; a < Pa; ++a) {
              if (!accept[a]) continue;
              T* Vb = V + (long long)off[a] * n;
              gemm1<T>(st, OP_N, OP_N, n, sz[a], sz[a], one, Vb, n, Qf + a * nbb, nb, zer, Vt, n, 0, 0, GS_EIG);
              axpby<T>(st, n, sz[a], 1.0, Vt, n, 0, 0.0, Vb, n, 0, 1);
            }
          }
          cand.swap(retry);
        }
        if (debug) {
          ZCSD_CUDA(cudaStreamSynchronize(st));
          fprintf(stderr, "zolo-eig: depth=%d group nb=%d blocks=%d attempt=%d: %.1f ms\n", depth, nb, Pa, attempt,
                  std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tg0).count());
        }
        ar.release(mg);
      }
      ar.release(matt);
    }
    for (const SplitState& w : work) {
      if (!w.done) {
        ed->status = CSD_ERR_EIG_SPLIT;
        throw EigFail{ed->splits, ed->retries};
      }
    }
    ar.release(mlev);
  }
  // ---- leaves: batched two-sided Jacobi on every block <= eig_leaf; scalar
  // blocks keep their diagonal
  std::vector<int> jo, js;
  for (size_t i = 0; i < leaf_off.size(); ++i) {
    if (leaf_sz[i] > 0) { jo.push_back(leaf_off[i]); js.push_back(leaf_sz[i]); }
    else diag_real<T>(st, -leaf_sz[i], Bw + leaf_off[i] + (long long)leaf_off[i] * n, n, lamw + leaf_off[i]);
  }
  const int nl = (int)jo.size();
  ed->leaves = nl;
  if (nl > 0) {
    const size_t ml = ar.mark();
    long long vtot = 0;
    for (int i = 0; i < nl; ++i) vtot += (long long)js[i] * js[i];
    T* Vl = ar.get<T>((size_t)vtot);
    std::vector<long long> voff;
    jacobi_eig_leaves<T>(cx, ar, jo, js, Bw, n, lamw, Vl, voff);
    for (int i = 0; i < nl; ++i) {
      gemm1<T>(st, OP_N, OP_N, n, js[i], js[i], one, V + (long long)jo[i] * n, n, Vl + voff[i], js[i], zer, Vt, n, 0,
               0, GS_EIG);
      axpby<T>(st, n, js[i], 1.0, Vt, n, 0, 0.0, V + (long long)jo[i] * n, n, 0, 1);
    }
    ar.release(ml);
  }
  // ---- sort the computed eigenpairs [lo, n) ascending
  const int cnt = n - lo;
  if (cnt > 0) {
    sort_perm(st, cnt, lamw + lo, perm);
    gather_vec(st, cnt, lamw + lo, perm, lam + lo);
    gather_cols<T>(st, n, cnt, V + (long long)lo * n, n, perm, Vt, n);
    axpby<T>(st, n, cnt, 1.0, Vt, n, 0, 0.0, V + (long long)lo * n, n, 0, 1);
  }
  if (lo > 0) ZCSD_CUDA(cudaMemsetAsync(lam, 0, sizeof(double) * lo, st));
  *lo_out = lo;
  ar.release(mk);
}

template void heig_impl<double>(Ctx&, Arena&, int, const double*, int, double*, double*, double, int*, EigDiag*);
template void heig_impl<z64>(Ctx&, Arena&, int, const z64*, int, double*, z64*, double, int*, EigDiag*);

}  // namespace zcsd
