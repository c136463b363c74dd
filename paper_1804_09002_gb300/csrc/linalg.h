// Blocked factorizations built from the kernels of blas.cu / fact.cu, and the
// device workspace arena they draw from.  Host-side orchestration only.
#pragma once
#include <algorithm>
#include <vector>

#include "ops.h"

namespace zcsd {

constexpr int NB_QR = 32;    // Householder panel width
constexpr int NB_OUT = 128;  // outer block of the two-level blocked QR
constexpr int NB_CHOL = 64;  // Cholesky / TRSM block size
constexpr int LEAF = 256;    // Zolo-eig leaf size (Jacobi), default
constexpr int LEAF_MAX = 1024;  // largest leaf size a context may set

struct ArenaOverflow {
  size_t needed;
};

// Bump allocator over one device allocation, with stack-like mark/release.
struct Arena {
  char* base = nullptr;
  size_t cap = 0, off = 0, peak = 0;
  template <class X>
  X* get(size_t count) {
    size_t bytes = (count * sizeof(X) + 255) & ~(size_t)255;
    if (off + bytes > cap) throw ArenaOverflow{off + bytes};
    X* p = reinterpret_cast<X*>(base + off);
    off += bytes;
    peak = std::max(peak, off);
    return p;
  }
  size_t mark() const { return off; }
  void release(size_t m) { off = m; }
};

// Pinned host scratch for device->host scalars.
struct HostScalars {
  double* d = nullptr;  // pinned, 64 doubles
  int* i = nullptr;     // pinned, 4096 ints
};

// ---- Householder QR of `batch` m x n matrices M_b (ld ldm, stride sM) in
// which the reflector of column k spans rows [k, min(m, k + band)).  On
// return M holds R (upper) and the reflectors (below); QRStore keeps the
// explicit V panels and T factors for applying / forming Q.
template <class T>
struct QRStore {
  int m = 0, n = 0, band = 0, batch = 0, npan = 0, ldy = 0, nbo = 0;
  int xrows = 0;    // rows [0, xrows) form the dense block X of a stacked [X; sqrt(c) I] (0: not stacked)
  T* Y = nullptr;  // per problem: npan outer blocks of ldy x nbo (nbo = min(NB_OUT, n rounded up to 32))
  T* Tf = nullptr; // per problem: npan blocks of nbo x nbo
  long long sY = 0, sT = 0;
};

template <class T> QRStore<T> qr_alloc(Arena& ar, int m, int n, int band, int batch);
template <class T> void qr_factor(cudaStream_t st, Arena& ar, QRStore<T>& q, T* M, int ldm, long long sM);
// E_b = Q_b [I; 0] (m x n, ld lde, stride sE)
template <class T> void qr_form_q(cudaStream_t st, Arena& ar, const QRStore<T>& q, T* E, int lde, long long sE);

// ---- upper Cholesky R^* R = Z_b (in place, upper triangle) of `batch` n x n
// matrices; Rinv receives the inverses of the NB_CHOL diagonal blocks
// (per problem NB_CHOL x n, block k at column k*NB_CHOL).  info[b] != 0 on a
// non-positive pivot.
template <class T>
void cholesky(cudaStream_t st, int n, T* Z, int ldz, long long sZ, T* Rinv, long long sR, int* info, int batch);

// ---- Tt_b = X_{b / xdiv} (R_b^* R_b)^{-1}: Yt = X R^{-1}, then Tt = Yt R^{-*}.
template <class T>
void trsm_pair(cudaStream_t st, Arena& ar, int n, const T* X, int ldx, long long sX, int xdiv, const T* Z, int ldz,
               long long sZ, const T* Rinv, long long sR, T* Yt, T* Tt, int ldt, long long sT, int batch);

}  // namespace zcsd
