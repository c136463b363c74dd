// Many real FP64 CS decompositions of different sizes in one graph-captured
// launch (csd_batch_*).  The paper's only parallelism is between the two
// polar decompositions and the r terms of Zolo-pd (Section 3, remark (ii));
// here independent CSDs are batched as well:
//
//  * instances are grouped into buckets of padded size nb (a multiple of the
//    bucket granularity); inside a bucket every polar problem is the n x n
//    block embedded as diag(A_i, I): Zolo-pd's QR and Cholesky forms keep
//    that block structure exactly, so the padded problems return
//    diag(W_i, I) and one zolo_pd call serves both blocks of every CSD of
//    the bucket (the sync-free form: no host read between its launches);
//  * H_i = sym(W_i^* A_i) and B = H_2 - H_1 per instance (the padded part of
//    B is exactly zero), and every B of every bucket is one leaf of the
//    batched one-sided Jacobi eigensolver at its own size, with a fixed
//    number of sweeps and device-side convergence flags;
//  * C, S = diag(V^* H_i V), theta = atan2(S, C), U_i = W_i V by batched
//    products on the padded V, then one CTA per instance sorts its angles
//    and writes its columns into the packed outputs.
//
// Everything between the input and the output buffers is on one stream with
// no host synchronisation, so the whole batch is captured once into a CUDA
// graph and replayed.  An autotuner picks the bucket granularity and, per
// bucket, the product engine (FP64-pipe tiles or the tensor-core kernel) by
// timing each candidate once on the caller's data.
#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "../../include/zolo_csd.h"
#include "solver.h"
#include "tc_gemm.h"

namespace zcsd {

namespace {

constexpr int BATCH_MAX_N = 1024;
constexpr int BATCH_SWEEPS = 30;  // Jacobi sweeps of the leaves (converged leaves are skipped)

struct Bucket {
  int nb = 0;                    // padded size
  std::vector<int> inst;         // instance indices
  bool tc = false;               // products on the tensor cores
  // device tables (persistent region): per bucket problem p (instance inst[p])
  int* dn = nullptr;             // n_i
  long long* doff = nullptr;     // element offset of instance i in the packed matrices
  long long* dtoff = nullptr;    // offset of instance i in the packed theta
  LeafTable leaves;              // B_p at p nb^2 (ld nb), eigenvalues at p nb
};

// X[2p + w] = diag(A_w of instance p, I), nb x nb (w = 0: A1, 1: A2)
__global__ void pad_gather_kernel(int nb, int P, const int* n, const long long* off, const double* A1,
                                  const double* A2, double* X) {
  const long long nn = (long long)nb * nb;
  const int q = blockIdx.y;
  const int p = q >> 1, w = q & 1, ni = n[p];
  const double* src = (w ? A2 : A1) + off[p];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn; t += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(t % nb), c = (int)(t / nb);
    X[q * nn + t] = (r < ni && c < ni) ? src[r + (long long)c * ni] : (r == c ? 1.0 : 0.0);
  }
}

// V_pad[p] = [V_p 0; 0 0] from the packed leaf eigenvectors
__global__ void pad_vectors_kernel(int nb, const int* n, const long long* goff, const double* Vl, double* Vp) {
  const long long nn = (long long)nb * nb;
  const int p = blockIdx.y, ni = n[p];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn; t += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(t % nb), c = (int)(t / nb);
    Vp[p * nn + t] = (r < ni && c < ni) ? Vl[goff[p] + r + (long long)c * ni] : 0.0;
  }
}

// One CTA per instance: ascending order of its angles (ties by index), then
// theta, U1, U2, V1 in that column order into the packed outputs; status
// CSD_ERR_NOT_CONVERGED when the instance's Jacobi leaf still rotated in the
// last sweep, CSD_ERR_INTERNAL when an angle is not finite (a failed
// factorization).
__global__ void __launch_bounds__(256) sort_scatter_kernel(int nb, const int* n, const long long* off,
                                                           const long long* toff, const double* th, const double* U1t,
                                                           const double* U2t, const double* Vp, double* theta,
                                                           double* U1, double* U2, double* V1, int* status,
                                                           const int* inst, const int* leaf_done) {
  extern __shared__ double sth[];
  int* rank = (int*)(sth + BATCH_MAX_N);
  const int p = blockIdx.x, ni = n[p];
  const long long nn = (long long)nb * nb;
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int j = threadIdx.x; j < ni; j += blockDim.x) {
    double v = th[(long long)p * nb + j];
    if (!(v == v) || v > 10.0 || v < -10.0) bad = 1;
    sth[j] = v;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < ni; j += blockDim.x) {
    const double v = sth[j];
    int r = 0;
    for (int k = 0; k < ni; ++k) r += (sth[k] < v) || (sth[k] == v && k < j);
    rank[j] = r;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < ni; j += blockDim.x) theta[toff[p] + rank[j]] = sth[j];
  for (long long t = threadIdx.x; t < (long long)ni * ni; t += blockDim.x) {
    const int r = (int)(t % ni), j = (int)(t / ni);
    const long long dst = off[p] + r + (long long)rank[j] * ni, src = p * nn + r + (long long)j * nb;
    U1[dst] = U1t[src];
    U2[dst] = U2t[src];
    V1[dst] = Vp[src];
  }
  if (threadIdx.x == 0) status[inst[p]] = bad ? CSD_ERR_INTERNAL : (leaf_done[p] ? CSD_OK : CSD_ERR_NOT_CONVERGED);
}

}  // namespace

// The product engine of a bucket: the tensor-core kernel or FP64 tiles.
struct EngineScope {
  TcState prev;
  EngineScope(bool tc, Arena& ar, int* err) : prev(t_tc) {
    t_tc = TcState{};
    t_tc.enabled = tc;
    t_tc.sites = ~0u;
    t_tc.ar = &ar;
    t_tc.err = err;
  }
  ~EngineScope() { t_tc = prev; }
};

// One bucket of the batch, enqueued on the context stream with no host
// synchronisation.
void run_bucket(Ctx& cx, Arena& ar, Bucket& bk, const double* A1, const double* A2, double* U1, double* U2, double* V1,
                double* theta, int* status, const int* dinst, int* tc_err) {
  cudaStream_t st = cx.stream;
  const int P = (int)bk.inst.size(), nb = bk.nb;
  const long long nn = (long long)nb * nb;
  const size_t mk = ar.mark();
  EngineScope eng(bk.tc, ar, tc_err);
  double* X = ar.get<double>(2 * P * nn);
  double* W = ar.get<double>(2 * P * nn);
  double* H = ar.get<double>(2 * P * nn);
  double* Bm = ar.get<double>(P * nn);
  double* lam = ar.get<double>((size_t)P * nb);
  double* G = ar.get<double>((size_t)bk.leaves.vtot);
  double* Vl = ar.get<double>((size_t)bk.leaves.vtot);
  double* Vp = ar.get<double>(P * nn);
  double* T1 = ar.get<double>(P * nn);
  double* T2 = ar.get<double>(P * nn);
  double* C = ar.get<double>((size_t)P * nb);
  double* S = ar.get<double>((size_t)P * nb);
  double* th = ar.get<double>((size_t)P * nb);
  const int gx = (int)std::min<long long>((nn + 255) / 256, 64);
  pad_gather_kernel<<<dim3(gx, 2 * P), 256, 0, st>>>(nb, P, bk.dn, bk.doff, A1, A2, X);
  ZCSD_LAUNCH();
  // lines 1-2 of Algorithm 1 for every block of every instance
  zolo_pd<double>(cx, ar, nb, 2 * P, X, W, nullptr, 0, 0, true);
  {
    GemmArgs<double> g;  // H = sym(W^* X)
    g.batch = 2 * P;
    g.m = nb; g.n = nb; g.k = nb; g.opA = OP_C; g.opB = OP_N;
    g.A = W; g.lda = nb; g.sA = nn;
    g.B = X; g.ldb = nb; g.sB = nn;
    g.C = H; g.ldc = nb; g.sC = nn;
    g.alpha = 1.0; g.beta = 0.0; g.site = GS_H;
    gemm(g, st);
    symmetrize<double>(st, nb, H, nb, nn, H, nb, nn, 2 * P);
  }
  // line 4: B = H2 - H1 (mu = 0)
  axpby<double>(st, nb, nb, 1.0, H + nn, nb, 2 * nn, 0.0, Bm, nb, nn, P);
  axpby<double>(st, nb, nb, -1.0, H, nb, 2 * nn, 1.0, Bm, nb, nn, P);
  // line 5: every B as one leaf of the batched Jacobi eigensolver
  leaf_solve<double>(cx, bk.leaves, Bm, lam, G, Vl, BATCH_SWEEPS);
  pad_vectors_kernel<<<dim3(gx, P), 256, 0, st>>>(nb, bk.dn, bk.leaves.goff, Vl, Vp);
  ZCSD_LAUNCH();
  // lines 6-9: C, S = diag(V^* H_i V), U_i = W_i V
  auto prod = [&](const double* A, long long sA, double* Cout, int site) {
    GemmArgs<double> g;
    g.batch = P;
    g.m = nb; g.n = nb; g.k = nb; g.opA = OP_N; g.opB = OP_N;
    g.A = A; g.lda = nb; g.sA = sA;
    g.B = Vp; g.ldb = nb; g.sB = nn;
    g.C = Cout; g.ldc = nb; g.sC = nn;
    g.alpha = 1.0; g.beta = 0.0; g.site = site;
    gemm(g, st);
  };
  prod(H, 2 * nn, T1, GS_ASSEMBLY);
  prod(H + nn, 2 * nn, T2, GS_ASSEMBLY);
  col_dots<double>(st, nb, P * nb, Vp, nb, T1, nb, C);
  col_dots<double>(st, nb, P * nb, Vp, nb, T2, nb, S);
  theta_from_cs(st, P * nb, C, S, th);
  prod(W, 2 * nn, T1, GS_ASSEMBLY);       // U1 (padded)
  prod(W + nn, 2 * nn, T2, GS_ASSEMBLY);  // U2 (padded)
  const size_t smem = BATCH_MAX_N * (sizeof(double) + sizeof(int));
  sort_scatter_kernel<<<P, 256, smem, st>>>(nb, bk.dn, bk.doff, bk.dtoff, th, T1, T2, Vp, theta, U1, U2, V1, status,
                                            dinst, bk.leaves.done);
  ZCSD_LAUNCH();
  ar.release(mk);
}

}  // namespace zcsd

using namespace zcsd;

struct csd_batch {
  csd_ctx* owner = nullptr;
  Ctx* cx = nullptr;
  int count = 0;
  std::vector<int> n;
  std::vector<long long> off, toff;
  int gran = 0;                         // chosen bucket granularity
  std::vector<Bucket> buckets;
  char* ws = nullptr;                   // persistent tables + run arena
  size_t ws_bytes = 0, persist_bytes = 0;
  int* dstatus = nullptr;               // per-instance status (device)
  int* dinst = nullptr;                 // bucket-order instance indices (device), per bucket at inst_off
  int* tc_err = nullptr;
  std::vector<int> inst_off;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  const void* bound[6] = {};            // buffers the captured graph reads / writes
  double tune_ms[3] = {0, 0, 0};        // autotuner: batch time per granularity (16, 32, 64)
  bool tuned = false;
  double ws_scale = 1.0;                // grows when a run overflows the arena
  size_t run_need = 0;                  // arena bytes a run was seen to need
  cudaStream_t stream = nullptr;        // the plan's own stream (tuning, capture, replay)
  cudaEvent_t ev = nullptr;
};

namespace {

size_t bucket_bytes(const Bucket& bk) {
  const long long P = (long long)bk.inst.size(), nb = bk.nb, nn = nb * nb;
  const size_t es = sizeof(double);
  size_t b = (size_t)(2 * P * nn * 3 + P * nn * 4 + P * nb * 4) * es + (size_t)bk.leaves.vtot * 2 * es;
  // zolo_pd on 2P problems plus the tensor-core slices of its largest product
  const long long r = R_MAX;
  const long long qr = 2 * (2 * nn) * 2 * P * r + (long long)ceil_div(nb, NB_OUT) * (nb + 1 + NB_OUT) * NB_OUT * 2 * P * r +
                       (long long)ceil_div(nb, NB_OUT) * NB_OUT * NB_OUT * 2 * P * r +
                       (long long)(5 * NB_OUT + (MAX_SUM + 1) * NB_QR) * nb * 2 * P * r;
  const long long ch = nn * 2 * P + 3 * nn * 2 * P * r + (long long)NB_CHOL * nb * 2 * P * r * (2 + MAX_SUM);
  b += (size_t)(2 * nn * 2 * P + std::max(qr, ch)) * es;
  b += (size_t)(2 * 14) * (nb + 128) * (2 * nb + 64) * 2 * P * r;  // BF16 slices of the stacked products
  return b + ((size_t)64 << 20);
}

void free_plan_ws(csd_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  if (b->ws) cudaFree(b->ws);
  b->ws = nullptr;
  b->ws_bytes = 0;
}

// Buckets for granularity `gran`, their device tables in the persistent
// region, and the workspace size.
int build_buckets(csd_batch* b, int gran) {
  free_plan_ws(b);
  b->gran = gran;
  std::map<int, std::vector<int>> by;
  for (int i = 0; i < b->count; ++i) by[ceil_div(b->n[i], gran) * gran].push_back(i);
  b->buckets.clear();
  for (auto& kv : by) {
    Bucket bk;
    bk.nb = kv.first;
    bk.inst = kv.second;
    bk.tc = false;
    b->buckets.push_back(bk);
  }
  // persistent region: per bucket n, off, toff and the leaf tables (index
  // arrays, shifts, one rotation record of 40 bytes per leaf row); statuses;
  // instance lists; every allocation rounded up to 256 bytes
  size_t pbytes = 0;
  for (auto& bk : b->buckets) {
    size_t rows = 0;
    for (int i : bk.inst) rows += (size_t)b->n[i];
    pbytes += bk.inst.size() * 128 + rows * 48 + 16 * 256;
  }
  pbytes += (size_t)b->count * 16 + 4 * 256 + (1 << 20);
  size_t run = 0;
  for (auto& bk : b->buckets) {
    long long vt = 0;
    for (int i : bk.inst) vt += (long long)b->n[i] * b->n[i];
    bk.leaves.vtot = vt;
    run = std::max(run, bucket_bytes(bk));
  }
  b->persist_bytes = (pbytes + 255) & ~(size_t)255;
  b->ws_bytes = b->persist_bytes + std::max((size_t)((double)run * b->ws_scale), b->run_need);
  if (cudaMalloc((void**)&b->ws, b->ws_bytes) != cudaSuccess) {
    cudaGetLastError();
    b->ws = nullptr;
    return CSD_ERR_ALLOC;
  }
  Ctx& cx = *b->cx;
  Arena per;
  per.base = b->ws;
  per.cap = b->persist_bytes;
  try {
    b->dstatus = per.get<int>(b->count);
    b->tc_err = per.get<int>(1);
    b->dinst = per.get<int>(b->count);
    b->inst_off.clear();
    std::vector<int> all;
    for (auto& bk : b->buckets) {
      b->inst_off.push_back((int)all.size());
      all.insert(all.end(), bk.inst.begin(), bk.inst.end());
      const int P = (int)bk.inst.size();
      std::vector<int> hn(P);
      std::vector<long long> ho(P), ht(P), boff(P);
      std::vector<int> lds(P, bk.nb), loff(P);
      for (int p = 0; p < P; ++p) {
        const int i = bk.inst[p];
        hn[p] = b->n[i];
        ho[p] = b->off[i];
        ht[p] = b->toff[i];
        boff[p] = (long long)p * bk.nb * bk.nb;
        loff[p] = p * bk.nb;
      }
      bk.dn = per.get<int>(P);
      bk.doff = per.get<long long>(P);
      bk.dtoff = per.get<long long>(P);
      ZCSD_CUDA(cudaMemcpyAsync(bk.dn, hn.data(), sizeof(int) * P, cudaMemcpyHostToDevice, cx.stream));
      ZCSD_CUDA(cudaMemcpyAsync(bk.doff, ho.data(), sizeof(long long) * P, cudaMemcpyHostToDevice, cx.stream));
      ZCSD_CUDA(cudaMemcpyAsync(bk.dtoff, ht.data(), sizeof(long long) * P, cudaMemcpyHostToDevice, cx.stream));
      bk.leaves = leaf_table_build(cx, per, boff, lds, loff, hn);
    }
    ZCSD_CUDA(cudaMemcpyAsync(b->dinst, all.data(), sizeof(int) * b->count, cudaMemcpyHostToDevice, cx.stream));
    ZCSD_CUDA(cudaStreamSynchronize(cx.stream));
  } catch (ArenaOverflow&) {
    return CSD_ERR_INTERNAL;
  } catch (CudaFail&) {
    return CSD_ERR_CUDA;
  }
  return CSD_OK;
}

// The whole batch on the context stream (capturable: no host sync).
void run_all(csd_batch* b, const double* A1, const double* A2, double* U1, double* U2, double* V1, double* theta) {
  Ctx& cx = *b->cx;
  Arena ar;
  ar.base = b->ws + b->persist_bytes;
  ar.cap = b->ws_bytes - b->persist_bytes;
  for (size_t k = 0; k < b->buckets.size(); ++k)
    run_bucket(cx, ar, b->buckets[k], A1, A2, U1, U2, V1, theta, b->dstatus, b->dinst + b->inst_off[k], b->tc_err);
}

// Per bucket engine choice, then the granularity with the smallest total.
int autotune(csd_batch* b, const double* A1, const double* A2, double* U1, double* U2, double* V1, double* theta) {
  const int grans[3] = {16, 32, 64};
  double best_total = 1e300;
  int best_g = 32;
  std::vector<char> best_tc;
  for (int gi = 0; gi < 3; ++gi) {
    int st = build_buckets(b, grans[gi]);
    if (st) return st;
    double total = 0.0;
    std::vector<char> choice;
    for (auto& bk : b->buckets) {
      Ctx& cx = *b->cx;
      Arena ar;
      ar.base = b->ws + b->persist_bytes;
      ar.cap = b->ws_bytes - b->persist_bytes;
      float ms[2];
      for (int e = 0; e < 2; ++e) {
        bk.tc = e == 1;
        const int* dinst = b->dinst + b->inst_off[&bk - &b->buckets[0]];
        run_bucket(cx, ar, bk, A1, A2, U1, U2, V1, theta, b->dstatus, dinst, b->tc_err);  // warm
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, cx.stream);
        run_bucket(cx, ar, bk, A1, A2, U1, U2, V1, theta, b->dstatus, dinst, b->tc_err);
        cudaEventRecord(e1, cx.stream);
        ZCSD_CUDA(cudaEventSynchronize(e1));
        cudaEventElapsedTime(&ms[e], e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
      }
      bk.tc = ms[1] < ms[0];
      choice.push_back(bk.tc);
      total += std::min(ms[0], ms[1]);
    }
    b->tune_ms[gi] = total;
    if (total < best_total) {
      best_total = total;
      best_g = grans[gi];
      best_tc = choice;
    }
  }
  int st = build_buckets(b, best_g);
  if (st) return st;
  for (size_t k = 0; k < b->buckets.size(); ++k) b->buckets[k].tc = best_tc[k];
  b->tuned = true;
  return CSD_OK;
}

}  // namespace


// Access to the context behind the opaque handle (solver.cu defines it).
zcsd::Ctx* ctx_internal(csd_ctx* ctx);

int csd_batch_create(csd_ctx* ctx, int count, const int* n, csd_batch** plan) {
  if (!ctx) return -1;
  if (count < 1) return -2;
  if (!n) return -3;
  if (!plan) return -4;
  for (int i = 0; i < count; ++i)
    if (n[i] < 1 || n[i] > BATCH_MAX_N) return -3;
  csd_batch* b = new (std::nothrow) csd_batch();
  if (!b) return CSD_ERR_ALLOC;
  b->owner = ctx;
  b->cx = ctx_internal(ctx);
  b->count = count;
  b->n.assign(n, n + count);
  b->off.assign(count + 1, 0);
  b->toff.assign(count + 1, 0);
  for (int i = 0; i < count; ++i) {
    b->off[i + 1] = b->off[i] + (long long)n[i] * n[i];
    b->toff[i + 1] = b->toff[i] + n[i];
  }
  *plan = b;
  return CSD_OK;
}

int csd_batch_run(csd_batch* b, const double* A1, const double* A2, double* U1, double* U2, double* V1,
                  double* theta, int* status) {
  if (!b) return -1;
  if (!A1) return -2;
  if (!A2) return -3;
  if (!U1) return -4;
  if (!U2) return -5;
  if (!V1) return -6;
  if (!theta) return -7;
  Ctx& cx = *b->cx;
  if (cudaSetDevice(cx.device) != cudaSuccess) {
    cudaGetLastError();
    return CSD_ERR_CUDA;
  }
  struct ProfOff {
    Profiler* prev;
    ProfOff() : prev(t_prof) { t_prof = nullptr; }
    ~ProfOff() { t_prof = prev; }
  } prof_off;
  // the batch runs on the plan's own non-blocking stream (a capture needs a
  // stream other than the legacy default one), ordered after the work
  // already queued on the context's stream and before whatever follows it
  if (!b->stream) {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return CSD_ERR_CUDA;
    }
  }
  struct StreamSwap {
    Ctx& c;
    cudaStream_t prev;
    StreamSwap(Ctx& c_, cudaStream_t s) : c(c_), prev(c_.stream) { c.stream = s; }
    ~StreamSwap() { c.stream = prev; }
  };
  if (cudaEventRecord(b->ev, cx.stream) != cudaSuccess || cudaStreamWaitEvent(b->stream, b->ev, 0) != cudaSuccess) {
    cudaGetLastError();
    return CSD_ERR_CUDA;
  }
  StreamSwap swap(cx, b->stream);
  for (int attempt = 0;; ++attempt) {
   try {
    if (!b->tuned) {
      const int st = autotune(b, A1, A2, U1, U2, V1, theta);
      if (st) return st;
    }
    const void* want[6] = {A1, A2, U1, U2, V1, theta};
    if (!b->exec || std::memcmp(want, b->bound, sizeof(want)) != 0) {
      if (b->exec) cudaGraphExecDestroy(b->exec);
      if (b->graph) cudaGraphDestroy(b->graph);
      b->exec = nullptr;
      b->graph = nullptr;
      ZCSD_CUDA(cudaMemsetAsync(b->tc_err, 0, sizeof(int), cx.stream));
      run_all(b, A1, A2, U1, U2, V1, theta);  // uncaptured once: lazy set-up outside the capture
      ZCSD_CUDA(cudaStreamSynchronize(cx.stream));
      ZCSD_CUDA(cudaStreamBeginCapture(cx.stream, cudaStreamCaptureModeThreadLocal));
      run_all(b, A1, A2, U1, U2, V1, theta);
      ZCSD_CUDA(cudaStreamEndCapture(cx.stream, &b->graph));
      ZCSD_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
      std::memcpy(b->bound, want, sizeof(want));
    }
    ZCSD_CUDA(cudaMemsetAsync(b->tc_err, 0, sizeof(int), cx.stream));
    ZCSD_CUDA(cudaGraphLaunch(b->exec, cx.stream));
    ZCSD_CUDA(cudaStreamSynchronize(cx.stream));
    int err = 0;
    ZCSD_CUDA(cudaMemcpy(&err, b->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (status) ZCSD_CUDA(cudaMemcpy(status, b->dstatus, sizeof(int) * b->count, cudaMemcpyDeviceToHost));
    if (err) return CSD_ERR_DEVICE_TIMEOUT;
    return CSD_OK;
   } catch (ArenaOverflow& o) {
    // a run needed more workspace than estimated: grow it and redo the set-up
    cudaStreamCaptureStatus cs;
    if (cudaStreamIsCapturing(cx.stream, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(cx.stream, &g);
      if (g) cudaGraphDestroy(g);
    }
    cudaStreamSynchronize(cx.stream);
    cudaGetLastError();
    if (attempt >= 6) return CSD_ERR_INTERNAL;
    b->ws_scale *= 2.0;
    b->run_need = std::max(b->run_need, o.needed + o.needed / 4);
    std::vector<char> tcs;
    for (auto& bk : b->buckets) tcs.push_back(bk.tc);
    const bool tuned = b->tuned;
    const int st = build_buckets(b, b->gran ? b->gran : 32);
    if (st) return st;
    for (size_t k = 0; k < b->buckets.size() && k < tcs.size(); ++k) b->buckets[k].tc = tcs[k];
    b->tuned = tuned;
    std::memset(b->bound, 0, sizeof(b->bound));
    continue;
   } catch (CudaFail& f) {
    fprintf(stderr, "zolo_csd: CUDA error %s at %s:%d\n", cudaGetErrorString(f.err), f.file, f.line);
    cudaStreamCaptureStatus cs;
    if (cudaStreamIsCapturing(cx.stream, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(cx.stream, &g);
      if (g) cudaGraphDestroy(g);
    }
    cudaGetLastError();
    return CSD_ERR_CUDA;
   }
  }
}

int csd_batch_destroy(csd_batch* b) {
  if (!b) return CSD_OK;
  cudaSetDevice(b->cx->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  free_plan_ws(b);
  if (b->ev) cudaEventDestroy(b->ev);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
  return CSD_OK;
}

int csd_batch_stats(const csd_batch* b, int* granularity, int* buckets, int* tc_buckets, double* tune_ms) {
  if (!b) return -1;
  if (granularity) *granularity = b->gran;
  if (buckets) *buckets = (int)b->buckets.size();
  if (tc_buckets) {
    int c = 0;
    for (auto& bk : b->buckets) c += bk.tc;
    *tc_buckets = c;
  }
  if (tune_ms)
    for (int i = 0; i < 3; ++i) tune_ms[i] = b->tune_ms[i];
  return CSD_OK;
}
