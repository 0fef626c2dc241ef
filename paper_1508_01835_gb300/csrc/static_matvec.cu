// static_matvec.cu -- fmm_matvec_static: the FMM product y = A_n x without any
// device allocation.
//
// Some callers cannot allocate device memory while they run: a host
// application that owns a fixed device pool and forbids further cudaMalloc,
// or a real-time loop that must not stall on the allocator.  For them this
// entry point takes its scratch (the multipole / local coefficients and x, y
// in tree order) from one file-scope device array of STATIC_SCRATCH_BYTES,
// which every GPU that loads the library holds until the process exits.  The
// caller passes x and y; the system's operators and lists (allocated when the
// system was created) are read in place.
//
// Set-up: the first call on a device looks up the array's device address with
// cudaGetSymbolAddress while that device is current; make that first call
// before any stream capture.  All calls share the array and it keeps the last
// call's contents; calls that overlap on the GPU race with each other.  No
// part of the array has to start at zero: each call writes every coefficient
// before reading it.  The tree lists the kernels walk are copied to the device
// once, when the system is created (build_static_lists), so a call copies
// nothing from the host and does no per-call host work beyond its launches.
#include <cstring>
#include <map>
#include <mutex>

#include "system.cuh"

namespace ifmm {

constexpr size_t STATIC_SCRATCH_BYTES = size_t(64) << 20;
static __device__ __align__(256) unsigned char g_static_scratch[STATIC_SCRATCH_BYTES];

static unsigned char* static_scratch(int device) {
  static std::mutex mu;
  static std::map<int, unsigned char*> addr;
  std::lock_guard<std::mutex> g(mu);
  auto it = addr.find(device);
  if (it != addr.end()) return it->second;
  void* p = nullptr;
  CK(cudaGetSymbolAddress(&p, g_static_scratch));
  addr[device] = static_cast<unsigned char*>(p);
  return static_cast<unsigned char*>(p);
}

// Per-depth view: the system's lists and this call's coefficients (in the array).
struct SLevel {
  const int* child_begin;  // nb + 1: children of box p are [child_begin[p], child_begin[p+1])
  const int* cpos;         // nb: position of the box inside its parent (0 .. 2^D - 1)
  const int* parent;       // nb
  const int* far_ptr;      // nb + 1
  const int* far_idx;      // interaction list entries
  const int* far_off;      // M2L table offset of each entry
  const double* m2l;       // M2L table of this depth
  double* mult;            // nb x nd x nrhs (column stride nb * nd)
  double* loc;
  int nb;
};

struct SLeaf {
  const int* p0;            // nb + 1 point offsets (tree order)
  const long long* uoff;    // nb: offset of U_i
  const int* nbr_ptr;       // nb + 1
  const int* nbr_idx;
  const long long* p2p_off; // per neighbour entry
  const double* U;
  const double* S;
  int nb;
};

// P2M: mult_L[i] = U_i^T x_i
__global__ void k_static_p2m(SLeaf lf, SLevel L, int nd, const double* __restrict__ x, long long N,
                             int nrhs) {
  const int i = blockIdx.x;
  const int p0 = lf.p0[i], m = lf.p0[i + 1] - p0;
  const double* U = lf.U + lf.uoff[i];
  const long long ldm = (long long)L.nb * nd;
  for (int c = 0; c < nrhs; c++)
    for (int r = threadIdx.x; r < nd; r += blockDim.x) {
      double s = 0.0;
      for (int q = 0; q < m; q++) s += U[q + (long long)r * m] * x[p0 + q + c * N];
      L.mult[(long long)i * nd + r + c * ldm] = s;
    }
}

// M2M: mult_l[p] = sum_children T_c^T mult_{l+1}[c]
__global__ void k_static_m2m(SLevel P, SLevel C, const double* __restrict__ T, int nd, int nrhs) {
  const int p = blockIdx.x;
  const long long ldp = (long long)P.nb * nd, ldc = (long long)C.nb * nd;
  for (int c = 0; c < nrhs; c++)
    for (int r = threadIdx.x; r < nd; r += blockDim.x) {
      double s = 0.0;
      for (int ch = P.child_begin[p]; ch < P.child_begin[p + 1]; ch++) {
        const double* Tc = T + (size_t)C.cpos[ch] * nd * nd;
        const double* y = C.mult + (long long)ch * nd + c * ldc;
        for (int q = 0; q < nd; q++) s += Tc[q + (long long)r * nd] * y[q];
      }
      P.mult[(long long)p * nd + r + c * ldp] = s;
    }
}

// M2L + L2L: loc_l[i] = sum_{q in I_i} K_iq mult_l[q] + T_i loc_{l-1}[parent(i)]
__global__ void k_static_m2l(SLevel L, SLevel P, const double* __restrict__ T, int nd, int nrhs,
                             int has_parent) {
  const int i = blockIdx.x;
  const long long ldl = (long long)L.nb * nd, ldp = (long long)P.nb * nd;
  for (int c = 0; c < nrhs; c++)
    for (int r = threadIdx.x; r < nd; r += blockDim.x) {
      double s = 0.0;
      for (int e = L.far_ptr[i]; e < L.far_ptr[i + 1]; e++) {
        const double* K = L.m2l + (size_t)L.far_off[e] * nd * nd;
        const double* y = L.mult + (long long)L.far_idx[e] * nd + c * ldl;
        for (int q = 0; q < nd; q++) s += K[r + (long long)q * nd] * y[q];
      }
      if (has_parent) {
        const double* Tc = T + (size_t)L.cpos[i] * nd * nd;
        const double* z = P.loc + (long long)L.parent[i] * nd + c * ldp;
        for (int q = 0; q < nd; q++) s += Tc[r + (long long)q * nd] * z[q];
      }
      L.loc[(long long)i * nd + r + c * ldl] = s;
    }
}

// L2P + P2P: y_i = U_i loc_L[i] + sum_{j in N_i} S_ij x_j
__global__ void k_static_l2p(SLeaf lf, SLevel L, int nd, const double* __restrict__ x,
                             double* __restrict__ y, long long N, int nrhs) {
  const int i = blockIdx.x;
  const int p0 = lf.p0[i], m = lf.p0[i + 1] - p0;
  const double* U = lf.U + lf.uoff[i];
  const long long ldl = (long long)L.nb * nd;
  for (int c = 0; c < nrhs; c++)
    for (int r = threadIdx.x; r < m; r += blockDim.x) {
      double s = 0.0;
      const double* z = L.loc + (long long)i * nd + c * ldl;
      for (int q = 0; q < nd; q++) s += U[r + (long long)q * m] * z[q];
      for (int e = lf.nbr_ptr[i]; e < lf.nbr_ptr[i + 1]; e++) {
        const int j = lf.nbr_idx[e];
        const int pj = lf.p0[j], mj = lf.p0[j + 1] - pj;
        const double* S = lf.S + lf.p2p_off[e];
        for (int q = 0; q < mj; q++) s += S[r + (long long)q * m] * x[pj + q + c * N];
      }
      y[p0 + r + c * N] = s;
    }
}

// Bump layout of the static array; every block 256-byte aligned.
struct Carver {
  unsigned char* base;
  size_t off = 0;
  template <class T>
  T* take(size_t n) {
    T* p = reinterpret_cast<T*>(base + off);
    off += (n * sizeof(T) + 255) & ~size_t(255);
    return p;
  }
};

// The lists of every depth, packed into one block of the system's memory.
void build_static_lists(ifmm_system* sys, cudaStream_t s) {
  const int L = sys->L, dim = sys->dim;
  std::vector<unsigned char> img;
  auto put = [&](const void* src, size_t n, size_t elem) {
    const size_t off = img.size();
    img.resize(off + ((n * elem + 255) & ~size_t(255)), 0);
    if (n) std::memcpy(img.data() + off, src, n * elem);
    return off;
  };
  struct Off { size_t cb, cpos, par, fptr, fidx, foff; };
  std::vector<Off> lo(L + 1);
  for (int l = 2; l <= L; l++) {
    const LevelTopo& v = sys->lv[l];
    std::vector<int> cb(v.nb + 1), cpos(v.nb), par(v.nb), foff(v.far.size());
    for (int p = 0; p < v.nb; p++) cb[p] = (l < L) ? v.cb[p] : 0;
    cb[v.nb] = (l < L) ? (v.nb ? v.ce[v.nb - 1] : 0) : 0;
    for (int i = 0; i < v.nb; i++) {
      cpos[i] = v.child_pos(i, dim);
      par[i] = v.parent.empty() ? 0 : v.parent[i];
      for (int e = v.far_ptr[i]; e < v.far_ptr[i + 1]; e++) foff[e] = v.m2l_offset(i, v.far[e], dim);
    }
    lo[l].cb = put(cb.data(), cb.size(), 4);
    lo[l].cpos = put(cpos.data(), cpos.size(), 4);
    lo[l].par = put(par.data(), par.size(), 4);
    lo[l].fptr = put(v.far_ptr.data(), v.far_ptr.size(), 4);
    lo[l].fidx = put(v.far.data(), v.far.size(), 4);
    lo[l].foff = put(foff.data(), foff.size(), 4);
  }
  const LevelTopo& leaf = sys->lv[L];
  std::vector<int> p0(leaf.nb + 1);
  for (int i = 0; i < leaf.nb; i++) p0[i] = leaf.p0[i];
  p0[leaf.nb] = (int)sys->N;
  const ChebOps& ops = sys->mv();
  const size_t o_p0 = put(p0.data(), p0.size(), 4);
  const size_t o_uoff = put(ops.uoff.data(), ops.uoff.size(), 8);
  const size_t o_nptr = put(leaf.nbr_ptr.data(), leaf.nbr_ptr.size(), 4);
  const size_t o_nidx = put(leaf.nbr.data(), leaf.nbr.size(), 4);
  const size_t o_p2p = put(sys->p2p_off.data(), sys->p2p_off.size(), 8);
  unsigned char* d = sys->mem.alloc<unsigned char>(std::max<size_t>(img.size(), 256));
  CK(cudaMemcpyAsync(d, img.data(), img.size(), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));  // img is a local
  sys->static_lv.assign(L + 1, StaticLevelLists{});
  for (int l = 2; l <= L; l++) {
    StaticLevelLists& q = sys->static_lv[l];
    q.child_begin = (const int*)(d + lo[l].cb);
    q.cpos = (const int*)(d + lo[l].cpos);
    q.parent = (const int*)(d + lo[l].par);
    q.far_ptr = (const int*)(d + lo[l].fptr);
    q.far_idx = (const int*)(d + lo[l].fidx);
    q.far_off = (const int*)(d + lo[l].foff);
  }
  sys->static_leaf.p0 = (const int*)(d + o_p0);
  sys->static_leaf.uoff = (const long long*)(d + o_uoff);
  sys->static_leaf.nbr_ptr = (const int*)(d + o_nptr);
  sys->static_leaf.nbr_idx = (const int*)(d + o_nidx);
  sys->static_leaf.p2p_off = (const long long*)(d + o_p2p);
}

void system_matvec_static(ifmm_system* sys, const double* x, double* y, int nrhs, long long ld,
                          int device, cudaStream_t s) {
  if (nrhs <= 0) return;
  if (sys->L == 0) {  // one dense block: the direct product needs no scratch
    launch_direct(sys->ks, sys->dim, sys->pts_user, sys->N, x, ld, y, ld, nrhs, s);
    return;
  }
  const ChebOps& ops = sys->mv();
  const int nd = ops.nd, L = sys->L;
  const long long N = sys->N;
  // scratch: multipole and local coefficients of every depth, x and y in tree order
  size_t bytes = 0;
  auto need = [&](size_t n) { bytes += (n * sizeof(double) + 255) & ~size_t(255); };
  for (int l = 2; l <= L; l++) {
    need((size_t)sys->lv[l].nb * nd * nrhs);  // mult
    need((size_t)sys->lv[l].nb * nd * nrhs);  // loc
  }
  need((size_t)N * nrhs);  // x in tree order
  need((size_t)N * nrhs);  // y in tree order
  if (bytes > STATIC_SCRATCH_BYTES)
    throw Error(IFMM_ERR_INVALID_ARG,
                "fmm_matvec_static: this system and nrhs need " + std::to_string(bytes) +
                    " bytes of scratch; the static buffer holds " +
                    std::to_string(STATIC_SCRATCH_BYTES) + " (use fewer right-hand sides or fmm_matvec)");
  Carver cv{static_scratch(device)};
  std::vector<SLevel> SL(L + 1);
  for (int l = 2; l <= L; l++) {
    SLevel& q = SL[l];
    const StaticLevelLists& g = sys->static_lv[l];
    q.nb = sys->lv[l].nb;
    q.child_begin = g.child_begin;
    q.cpos = g.cpos;
    q.parent = g.parent;
    q.far_ptr = g.far_ptr;
    q.far_idx = g.far_idx;
    q.far_off = g.far_off;
    q.m2l = ops.m2l[l];
    q.mult = cv.take<double>((size_t)q.nb * nd * nrhs);
    q.loc = cv.take<double>((size_t)q.nb * nd * nrhs);
  }
  const LevelTopo& leaf = sys->lv[L];
  SLeaf lf;
  lf.nb = leaf.nb;
  lf.p0 = sys->static_leaf.p0;
  lf.uoff = sys->static_leaf.uoff;
  lf.nbr_ptr = sys->static_leaf.nbr_ptr;
  lf.nbr_idx = sys->static_leaf.nbr_idx;
  lf.p2p_off = sys->static_leaf.p2p_off;
  lf.U = ops.leafU;
  lf.S = sys->p2p;
  double* xt = cv.take<double>((size_t)N * nrhs);
  double* yt = cv.take<double>((size_t)N * nrhs);
  launch_gather_rows(sys->perm, N, x, ld, xt, N, nrhs, s);
  k_static_p2m<<<leaf.nb, 64, 0, s>>>(lf, SL[L], nd, xt, N, nrhs);
  CK_LAUNCH("k_static_p2m");
  for (int l = L - 1; l >= 2; l--) {
    k_static_m2m<<<SL[l].nb, 64, 0, s>>>(SL[l], SL[l + 1], ops.transfer, nd, nrhs);
    CK_LAUNCH("k_static_m2m");
  }
  for (int l = 2; l <= L; l++) {
    k_static_m2l<<<SL[l].nb, 64, 0, s>>>(SL[l], SL[l > 2 ? l - 1 : l], ops.transfer, nd, nrhs,
                                         l > 2);
    CK_LAUNCH("k_static_m2l");
  }
  k_static_l2p<<<leaf.nb, 64, 0, s>>>(lf, SL[L], nd, xt, yt, N, nrhs);
  CK_LAUNCH("k_static_l2p");
  launch_scatter_rows(sys->perm, N, yt, N, y, ld, nrhs, s);
}

}  // namespace ifmm
