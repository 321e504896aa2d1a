// C ABI of the staggered-grid Navier-Stokes step: grid objects, device
// layout, boundary tables, stage orchestration and CUDA-graph replay.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "cfd_internal.h"
#include "gb300cfd.h"

using namespace cfd;

namespace {

// An NVTX range around one entry point (shows the library's calls on a
// profiler's timeline; a push and a pop are two inline checks when no tool
// is attached).
struct CallRange {
  explicit CallRange(const char* name) { nvtxRangePushA(name); }
  ~CallRange() { nvtxRangePop(); }
  CallRange(const CallRange&) = delete;
  CallRange& operator=(const CallRange&) = delete;
};

thread_local std::string t_err = "no error";

cfd_status fail(cfd_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  t_err = buf;
  return s;
}

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

const int kSets[3][3] = {{A_U, A_V, A_W}, {A_WU, A_WV, A_WW}, {A_U1, A_V1, A_W1}};

struct HostBlock {
  int n[3];
  int origin[3];
  int py;
  long long pz;
  long long planes;
  size_t array_bytes;
  size_t first_byte;     // byte offset of this block's first array from base
  int nbr[6];
};

}  // namespace

struct cfd_grid {
  int nblocks = 0, g = 1, dtype = CFD_F32, es = 4;
  double h[3] = {1, 1, 1};
  int gdims[3] = {0, 0, 0};
  bool blockset = false;
  std::vector<HostBlock> hb;
  std::vector<int> hn;  // nblocks x 3 dims (for grid sizing)
  int bc[6] = {0, 0, 0, 0, 0, 0};
  double wall[6][3] = {};
  double nu = 0.0, omega = 1.0;
  int iters = 50, order = 2;
  int form = CFD_ADVECTIVE;  // advection term (cfd_set_advection)

  cudaStream_t user = nullptr, own = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  int device = 0, sms = 1;

  char* base = nullptr;
  size_t bytes = 0;
  bool owns = false;
  size_t table_off = 0, items_off = 0, partial_off = 0, out_off = 0, flag_off = 0;
  size_t maps_off = 0;            // TMA tensor maps: nblocks x {P, P2, R}
  size_t adj_off = 0;             // adjoint scalars: [0] dL/dnu accumulator
  bool maps_ready = false;        // maps encoded for the current Jacobi config
  size_t arrays_off = 0;
  size_t staging_off = 0;         // contiguous interior of one array (host copies)
  int host_copy = CFD_HOST_COPY_KERNEL;  // route of page-locked host copies
  int nparts = 0;
  // ghost-fill work items: the grid's blocks first, then each multigrid
  // level's (gitem_first[l], gitem_count[l]; l = 0 the grid itself)
  std::vector<GhostItem> gitems;
  std::vector<int> gitem_first, gitem_count;
  std::vector<BlockDev> bdev;
  double* h_out = nullptr;  // pinned, 4 doubles
  int* h_flag = nullptr;    // pinned, 1 int

  double t = 0.0;
  long long step = 0;
  bool sticky = false;

  JacobiCfg jcfg{0, 4, 8, 32, 4};
  StencilCfg scfg{8, 32, 1};
  bool per_block = false;  // baseline mode: one launch per block per stencil kernel

  cudaGraphExec_t gexec = nullptr;
  bool graph_valid = false;
  double graph_dt = 0.0;
  long long graph_nodes = 0;   // kernel launches per replay
  long long launches = 0;      // kernel launches enqueued (incl. replays)

  // geometric multigrid (single FP32 block): coarse levels 1..mg_max, each
  // with three arrays (correction P, its ping-pong P2, residual R)
  struct MgLevel {
    int n[3];
    int py;
    long long pz;
    size_t array_bytes, first_byte;
  };
  std::vector<MgLevel> mgl;   // level l at index l - 1
  std::vector<BlockDev> mg_bdev;
  std::vector<int> mg_hn;     // 3 ints per level
  size_t mg_table_off = 0;
  int mg_levels = 0, mg_nu1 = 2, mg_nu2 = 2, mg_ncoarse = 30;  // mg_levels 0: all
  double mg_omega = 6.0 / 7.0;
  cudaGraphExec_t mg_exec = nullptr;  // one V-cycle, captured on first use
  bool mg_valid = false;
  long long mg_nodes = 0;
  int solver = CFD_SOLVER_JACOBI;  // pressure solve inside the step's stages
  int mg_cycles = 2;               // V-cycles per stage solve (CFD_SOLVER_MG)

  // rollout graphs: segment recompute and segment adjoint, keyed by length
  struct SegGraph { cudaGraphExec_t exec = nullptr; long long nodes = 0; int len = 0; };
  SegGraph rec_graph[2], adj_graph[2];
  const void* seg_store = nullptr;
  double seg_dt = 0.0;
  int seg_len = 0;
};

namespace {

cfd_status cuda_fail(cfd_grid* g, cudaError_t e, const char* what) {
  if (g) g->sticky = true;
  return fail(CFD_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(g, call)                                           \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail((g), e_, #call);  \
  } while (0)

cfd_status usable(cfd_grid* g) {
  if (!g) return fail(CFD_EINVAL, "null grid");
  if (g->sticky) return fail(CFD_ECUDA, "grid is in a failed state after an earlier CUDA error");
  if (!g->base) return fail(CFD_ESTATE, "no device memory bound (cfd_bind_memory / cfd_alloc_memory)");
  for (int d = 0; d < 3; ++d)
    if ((g->bc[2 * d] == CFD_BC_PERIODIC) != (g->bc[2 * d + 1] == CFD_BC_PERIODIC))
      return fail(CFD_EINVAL, "axis %d: periodic on one face but not the other", d);
  if (g->order == 4 && g->g < 2) return fail(CFD_EINVAL, "order 4 needs ghost width 2");
  return CFD_OK;
}

// Device layout: [tables][arrays of block 0][arrays of block 1]...
// The ghost-fill work items of blocks with dims n (3 ints each) and
// neighbours nbr (6 each), faces bc, ghost width gw, appended to out: per
// block the 26 boxes of its ghost shell with their sources (axis by axis,
// x then y then z: across a periodic face into the neighbour, mirrored at a
// wall), each cut into pieces of at most eight warp-wide steps (GhostItem).
// False if the grid has 2^30 or more pieces.
bool ghost_items(const int* n, const int* nbr, int nb, const int bc[6], int gw,
                 std::vector<GhostItem>& out) {
  for (int b = 0; b < nb; ++b)
    for (int dir = 0; dir < 27; ++dir) {
      if (dir == 13) continue;
      const int dv[3] = {dir % 3 - 1, (dir / 3) % 3 - 1, dir / 9 - 1};
      int ext[3], d0[3], s0[3], st[3], wf[3] = {-1, -1, -1};
      int sbk = b;
      for (int a = 0; a < 3; ++a) {
        const int N = n[3 * b + a];
        if (dv[a] == 0) {
          ext[a] = N;
          d0[a] = 0;
          s0[a] = 0;
          st[a] = 1;
          continue;
        }
        const int face = dv[a] < 0 ? 2 * a : 2 * a + 1;
        ext[a] = gw;
        d0[a] = dv[a] < 0 ? -gw : N;
        if (bc[face] == CFD_BC_PERIODIC) {  // into the neighbour (itself for one block)
          const int to = nbr[6 * sbk + face];
          s0[a] = dv[a] < 0 ? n[3 * to + a] - gw : 0;
          st[a] = 1;
          sbk = to;
        } else {  // mirror: ghost layer m takes the cell m - 1 from the wall
          s0[a] = dv[a] < 0 ? gw - 1 : N - 1;
          st[a] = -1;
          wf[a] = face;
        }
      }
      // inner axis x unless the box is one cell thin there (two ghost
      // layers side by side share a 32-byte sector, so one warp access
      // takes both); rows along the longer of the other two axes
      const int ia = ext[0] >= 2 ? 0 : (ext[1] >= ext[2] ? 1 : 2);
      const int o1 = ia == 0 ? 1 : 0, o2 = ia == 2 ? 1 : 2;
      const int ja = ext[o1] >= ext[o2] ? o1 : o2, ka = ja == o1 ? o2 : o1;
      const int ax[3] = {ia, ja, ka};
      const int ei = ext[ia], ej = ext[ja], ek = ext[ka];
      for (int i0 = 0; i0 < ei; i0 += kGhostItemCells) {
        const int ni = std::min(kGhostItemCells, ei - i0);
        int sh = 0;
        while ((1 << sh) < ni && sh < 5) ++sh;     // columns: ni rounded up to a power of two, <= 32
        const int passes = (ni + (1 << sh) - 1) >> sh;
        const int rows = (32 >> sh) * std::max(1, 8 / passes);  // rows of one piece
        for (int rk = 0; rk < ek; ++rk)
          for (int rj0 = 0; rj0 < ej; rj0 += rows) {
            GhostItem it{};
            it.dst = b;
            it.src = sbk;
            for (int k = 0; k < 3; ++k) {
              it.ax[k] = ax[k];
              it.d0[k] = d0[ax[k]];
              it.s0[k] = s0[ax[k]];
              it.st[k] = st[ax[k]];
              it.wface[k] = wf[k];
            }
            it.i0 = i0;
            it.ni = ni;
            it.rj0 = rj0;
            it.nrows = std::min(rows, ej - rj0);
            it.rk = rk;
            it.sh = sh;
            it.passes = passes;
            out.push_back(it);
            if (out.size() >= (size_t)1 << 30) return false;  // CTA numbers x 8 warps in 32 bits
          }
      }
    }
  return true;
}

// All ghost items of the grid and of its multigrid levels (gitems empty if
// there are too many).  Depends on the faces' kinds: rebuilt with the tables.
void build_ghost_items(cfd_grid* g) {
  g->gitems.clear();
  g->gitem_first.assign(g->mgl.size() + 1, 0);
  g->gitem_count.assign(g->mgl.size() + 1, 0);
  std::vector<int> n, nbr;
  for (const auto& b : g->hb) {
    n.insert(n.end(), b.n, b.n + 3);
    nbr.insert(nbr.end(), b.nbr, b.nbr + 6);
  }
  bool ok = ghost_items(n.data(), nbr.data(), g->nblocks, g->bc, g->g, g->gitems);
  g->gitem_count[0] = (int)g->gitems.size();
  const int self[6] = {0, 0, 0, 0, 0, 0};
  for (size_t l = 0; l < g->mgl.size() && ok; ++l) {
    g->gitem_first[l + 1] = (int)g->gitems.size();
    ok = ghost_items(g->mgl[l].n, self, 1, g->bc, g->g, g->gitems);
    g->gitem_count[l + 1] = (int)g->gitems.size() - g->gitem_first[l + 1];
  }
  if (!ok) g->gitems.clear();
}

void plan_layout(cfd_grid* g) {
  const int align_e = kAlignBytes / g->es;
  size_t off = 0;
  g->table_off = off;
  off = round_up(off + sizeof(BlockDev) * g->nblocks, 256);
  g->nparts = 8 * g->sms;  // reduction CTAs: 8 per SM of 256 threads (full occupancy)
  g->partial_off = off;
  off = round_up(off + sizeof(double) * 4 * g->nparts, 256);
  g->out_off = off;
  off = round_up(off + sizeof(double) * 4, 256);
  g->flag_off = off;
  off = round_up(off + 256, 256);
  g->maps_off = off;
  off = round_up(off + (size_t)kTmaMapBytes * 3 * g->nblocks, 256);
  g->adj_off = off;
  off = round_up(off + 8 * sizeof(double), 256);
  // multigrid levels: every axis halves while all are even and >= 4
  g->mgl.clear();
  if (g->nblocks == 1 && g->dtype == CFD_F32) {
    int n[3] = {g->hb[0].n[0], g->hb[0].n[1], g->hb[0].n[2]};
    while (g->mgl.size() < 16 && n[0] % 2 == 0 && n[1] % 2 == 0 && n[2] % 2 == 0 && n[0] >= 4 &&
           n[1] >= 4 && n[2] >= 4) {
      cfd_grid::MgLevel m{};
      for (int a = 0; a < 3; ++a) m.n[a] = (n[a] /= 2);
      g->mgl.push_back(m);
    }
  }
  const size_t nl = g->mgl.size();
  g->mg_table_off = off;
  off = round_up(off + sizeof(BlockDev) * std::max<size_t>(nl, 1), 256);
  // ghost items (their number depends on the dims and the ghost width only)
  build_ghost_items(g);
  g->items_off = off;
  off = round_up(off + sizeof(GhostItem) * std::max<size_t>(g->gitems.size(), 1), 256);
  g->arrays_off = off;
  for (auto& b : g->hb) {
    b.py = (int)round_up((size_t)align_e + b.n[0] + g->g, align_e);
    b.pz = (long long)b.py * (b.n[1] + 2 * g->g);
    b.planes = b.n[2] + 2 * g->g;
    b.array_bytes = round_up((size_t)b.pz * b.planes * g->es, 256);
    b.first_byte = off;
    off += b.array_bytes * kNumArrays;
  }
  // staging for host copies: the compact interior of the largest block
  size_t stage = 0;
  for (auto& b : g->hb)
    stage = std::max(stage, (size_t)b.n[0] * b.n[1] * b.n[2] * g->es);
  g->staging_off = off;
  off += round_up(stage, 256);
  g->mg_hn.clear();
  for (auto& m : g->mgl) {
    m.py = (int)round_up((size_t)align_e + m.n[0] + g->g, align_e);
    m.pz = (long long)m.py * (m.n[1] + 2 * g->g);
    m.array_bytes = round_up((size_t)m.pz * (m.n[2] + 2 * g->g) * g->es, 256);
    m.first_byte = off;
    off += 3 * m.array_bytes;
    for (int a = 0; a < 3; ++a) g->mg_hn.push_back(m.n[a]);
  }
  off += 256;  // tail pad: a 4-byte halo copy next to the very last row stays inside
  g->bytes = off;
}

void build_tables(cfd_grid* g) {
  const int align_e = kAlignBytes / g->es;
  build_ghost_items(g);  // same count as planned: the faces' kinds change only the sources
  g->bdev.resize(g->nblocks);
  for (int i = 0; i < g->nblocks; ++i) {
    const HostBlock& b = g->hb[i];
    BlockDev& d = g->bdev[i];
    memset(&d, 0, sizeof d);
    for (int a = 0; a < 3; ++a) d.n[a] = b.n[a];
    d.py = b.py;
    d.pz = b.pz;
    for (int a = 0; a < kNumArrays; ++a) {
      const size_t start = b.first_byte + b.array_bytes * a;
      d.org[a] = (long long)(start / g->es) + (long long)g->g * b.pz + (long long)g->g * b.py + align_e;
    }
    for (int f = 0; f < 6; ++f) {
      d.nbr[f] = b.nbr[f];
      d.bc[f] = g->bc[f];
      for (int c = 0; c < 3; ++c) d.wall[f][c] = (float)g->wall[f][c];
    }
  }
  // multigrid levels: one self-neighbouring block each; P, P2 and R are the
  // level's three arrays, the other ids alias P and are never addressed
  g->mg_bdev.resize(g->mgl.size());
  for (size_t l = 0; l < g->mgl.size(); ++l) {
    const auto& m = g->mgl[l];
    BlockDev& d = g->mg_bdev[l];
    memset(&d, 0, sizeof d);
    for (int a = 0; a < 3; ++a) d.n[a] = m.n[a];
    d.py = m.py;
    d.pz = m.pz;
    const long long lead = (long long)g->g * m.pz + (long long)g->g * m.py + align_e;
    for (int a = 0; a < kNumArrays; ++a) {
      const int slot = a == A_P2 ? 1 : a == A_R ? 2 : 0;
      d.org[a] = (long long)((m.first_byte + m.array_bytes * slot) / g->es) + lead;
    }
    for (int f = 0; f < 6; ++f) d.bc[f] = g->bc[f];
  }
}

cfd_status refresh_maps(cfd_grid* g);

cfd_status upload_tables(cfd_grid* g) {
  if (!g->base) return CFD_OK;
  build_tables(g);
  CK(g, cudaMemcpyAsync(g->base + g->table_off, g->bdev.data(), sizeof(BlockDev) * g->nblocks,
                        cudaMemcpyHostToDevice, g->own));
  CK(g, cudaMemcpyAsync(g->base + g->items_off, g->gitems.data(),
                        sizeof(GhostItem) * g->gitems.size(), cudaMemcpyHostToDevice, g->own));
  CK(g, cudaMemsetAsync(g->base + g->flag_off, 0, 256, g->own));
  if (!g->mgl.empty()) {
    CK(g, cudaMemcpyAsync(g->base + g->mg_table_off, g->mg_bdev.data(),
                          sizeof(BlockDev) * g->mg_bdev.size(), cudaMemcpyHostToDevice, g->own));

  }
  CK(g, cudaStreamSynchronize(g->own));
  return refresh_maps(g);
}

// Tensor maps of the TMA Jacobi sweep (box sizes depend on the config).
cfd_status refresh_maps(cfd_grid* g) {
  g->maps_ready = false;
  if ((g->jcfg.kind != 1 && g->jcfg.kind != 7 && g->jcfg.kind != 9) || !g->base) return CFD_OK;
  std::vector<TmaArray> arrs;
  const int ids[3] = {A_P, A_P2, A_R};
  for (const auto& b : g->hb)
    for (int a : ids)
      arrs.push_back(TmaArray{g->base + b.first_byte + b.array_bytes * a, b.py,
                              (long long)b.n[1] + 2 * g->g, b.planes});
  std::vector<unsigned char> host(arrs.size() * kTmaMapBytes + 64);
  unsigned char* aligned = host.data() + ((64 - (reinterpret_cast<uintptr_t>(host.data()) % 64)) % 64);
  if (!encode_jacobi_maps(aligned, arrs.data(), (int)arrs.size(), g->dtype, g->jcfg))
    return fail(CFD_EUNSUPPORTED, "TMA tensor map encoding failed for this Jacobi config");
  CK(g, cudaMemcpyAsync(g->base + g->maps_off, aligned, arrs.size() * kTmaMapBytes,
                        cudaMemcpyHostToDevice, g->own));
  CK(g, cudaStreamSynchronize(g->own));
  g->maps_ready = true;
  return CFD_OK;
}

Launch make_launch(cfd_grid* g) {
  Launch L;
  L.blocks = reinterpret_cast<const BlockDev*>(g->base + g->table_off);
  L.b0 = 0;
  L.nblocks = g->nblocks;
  L.base = g->base;
  L.dtype = g->dtype;
  L.ghost = g->g;
  for (int d = 0; d < 3; ++d) {
    L.ih[d] = (float)(1.0 / g->h[d]);
    L.ih2[d] = (float)(1.0 / (g->h[d] * g->h[d]));
  }
  L.err_flag = reinterpret_cast<int*>(g->base + g->flag_off);
  L.stream = g->own;
  L.sms = g->sms;
  L.hn = reinterpret_cast<const int(*)[3]>(g->hn.data());
  return L;
}

cfd_status common_init(cfd_grid* g, int ghost, const double h[3], int storage, void* stream) {
  if (ghost < 1 || ghost > kMaxGhost) return fail(CFD_EINVAL, "ghost width must be 1 or 2");
  if (!h) return fail(CFD_EINVAL, "null h");
  for (int d = 0; d < 3; ++d)
    if (!(h[d] > 0.0) || !std::isfinite(h[d])) return fail(CFD_EINVAL, "cell size h[%d] must be > 0", d);
  if (storage < CFD_F32 || storage > CFD_F16) return fail(CFD_EINVAL, "unknown storage dtype %d", storage);
  g->g = ghost;
  for (int d = 0; d < 3; ++d) g->h[d] = h[d];
  g->dtype = storage;
  g->es = storage == CFD_F32 ? 4 : 2;
  g->user = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e;
  if ((e = cudaGetDevice(&g->device)) != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDevice");
  if ((e = cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, g->device)) != cudaSuccess)
    return cuda_fail(nullptr, e, "cudaDeviceGetAttribute");
  if ((e = cudaStreamCreateWithFlags(&g->own, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_fail(nullptr, e, "cudaStreamCreate");
  if ((e = cudaEventCreateWithFlags(&g->ev_in, cudaEventDisableTiming)) != cudaSuccess)
    return cuda_fail(nullptr, e, "cudaEventCreate");
  if ((e = cudaEventCreateWithFlags(&g->ev_out, cudaEventDisableTiming)) != cudaSuccess)
    return cuda_fail(nullptr, e, "cudaEventCreate");
  if ((e = cudaMallocHost(&g->h_out, 8 * sizeof(double))) != cudaSuccess)
    return cuda_fail(nullptr, e, "cudaMallocHost");
  g->h_flag = reinterpret_cast<int*>(g->h_out + 4);
  g->hn.resize(3 * g->nblocks);
  for (int b = 0; b < g->nblocks; ++b)
    for (int d = 0; d < 3; ++d) g->hn[3 * b + d] = g->hb[b].n[d];
  g->jcfg = JacobiCfg{0, 4, 8, 32, 4};
  plan_layout(g);
  if (g->gitems.empty())  // the ghost kernel numbers its pieces in 32 bits
    return fail(CFD_EINVAL, "the ghost shell has 2^30 or more pieces");
  if (!g->mgl.empty() && (e = prepare_mg_bottom()) != cudaSuccess)
    return cuda_fail(nullptr, e, "cudaFuncSetAttribute");
  return CFD_OK;
}

void drop_seg_graphs(cfd_grid* g) {
  for (int q = 0; q < 2; ++q) {
    if (g->rec_graph[q].exec) cudaGraphExecDestroy(g->rec_graph[q].exec);
    if (g->adj_graph[q].exec) cudaGraphExecDestroy(g->adj_graph[q].exec);
    g->rec_graph[q] = cfd_grid::SegGraph();
    g->adj_graph[q] = cfd_grid::SegGraph();
  }
  g->seg_store = nullptr;
}

void destroy_handles(cfd_grid* g) {
  drop_seg_graphs(g);
  if (g->gexec) cudaGraphExecDestroy(g->gexec);
  if (g->mg_exec) cudaGraphExecDestroy(g->mg_exec);
  if (g->own) cudaStreamSynchronize(g->own);
  if (g->owns && g->base) cudaFree(g->base);
  if (g->h_out) cudaFreeHost(g->h_out);
  if (g->ev_in) cudaEventDestroy(g->ev_in);
  if (g->ev_out) cudaEventDestroy(g->ev_out);
  if (g->own) cudaStreamDestroy(g->own);
}

// Order the private stream after the caller's stream, and back.
cfd_status join_in(cfd_grid* g) {
  CK(g, cudaEventRecord(g->ev_in, g->user));
  CK(g, cudaStreamWaitEvent(g->own, g->ev_in, 0));
  return CFD_OK;
}
cfd_status join_out(cfd_grid* g) {
  CK(g, cudaEventRecord(g->ev_out, g->own));
  CK(g, cudaStreamWaitEvent(g->user, g->ev_out, 0));
  return CFD_OK;
}

// ------------------------------------------------------------- enqueuers

// Runs f(L) once over all blocks (one persistent launch walks the tiles of
// every block), or once per block in the per-block baseline mode.
template <typename F>
cfd_status each_launch(cfd_grid* g, F f) {
  Launch L = make_launch(g);
  if (!g->per_block) {
    CK(g, f(L));
    g->launches += 1;
    return CFD_OK;
  }
  for (int b = 0; b < g->nblocks; ++b) {
    Launch Lb = L;
    Lb.b0 = b;
    Lb.nblocks = 1;
    CK(g, f(Lb));
    g->launches += 1;
  }
  return CFD_OK;
}

cfd_status enq_ghost(cfd_grid* g, unsigned mask) {
  int arrs[kNumArrays];
  int n = 0;
  for (int a = 0; a < kNumArrays; ++a)
    if (mask & (1u << a)) arrs[n++] = a;
  const Launch L = make_launch(g);
  CK(g, launch_ghost(L, arrs, n, reinterpret_cast<const GhostItem*>(g->base + g->items_off),
                     g->gitem_count[0]));
  g->launches += n > 0 ? 1 : 0;
  return CFD_OK;
}

unsigned set_mask(int s) {
  return (1u << kSets[s][0]) | (1u << kSets[s][1]) | (1u << kSets[s][2]);
}

cfd_status enq_stage(cfd_grid* g, double a, int xs, double b, int ys, double c, int os) {
  return each_launch(g, [&](const Launch& L) {
    const int scheme = g->form == CFD_FLUX ? kSchemeFlux2 : g->order;
    return launch_stage(L, g->scfg, scheme, (float)a, a != 0.0 ? kSets[xs] : nullptr, (float)b,
                        kSets[ys], (float)c, kSets[os], (float)g->nu);
  });
}

// The two-sweep kernel's periodic form: every face periodic (or, in a block
// set, copied from the neighbouring block) and two ghost layers (the first
// sweep is also taken on the first ghost layer, whose cells the ghost launch
// before each two-sweep launch has copied from where they live).
bool ws2_periodic(const cfd_grid* g) {
  for (int f = 0; f < 6; ++f)
    if (g->bc[f] != CFD_BC_PERIODIC) return false;
  return g->g >= 2;
}

// Fused two-sweep launches apply: kind 9 on a single block whose six faces
// are walls, or in the periodic form (single blocks and block sets); kind 5
// on single blocks with tiles dividing x and y.  Never in the one-launch-
// per-block mode, whose sweeps are the baseline of the batched form.
bool fused_ok(const cfd_grid* g) {
  if (g->per_block && g->nblocks > 1) return false;
  if (g->jcfg.kind == 9) {
    if (!g->maps_ready) return false;
    if (ws2_periodic(g)) return true;
    if (g->nblocks != 1) return false;
    bool walls = true;
    for (int f = 0; f < 6; ++f) walls &= g->bdev[0].bc[f] == BC_WALL;
    return walls;
  }
  return g->jcfg.kind == 5 && g->nblocks == 1 && g->hb[0].n[0] % 128 == 0 &&
         g->hb[0].n[1] % g->jcfg.ty == 0 && g->hb[0].n[1] >= 2 && g->hb[0].n[2] >= 2;
}

// One Jacobi sweep src -> dst with the configured variant (the fused
// variant's single sweeps use the register/shuffle kernel).
cudaError_t sweep(cfd_grid* g, const Launch& L, int src, int dst, float omega) {
  if (g->jcfg.kind == 5 || g->jcfg.kind == 9)
    return launch_jacobi(L, JacobiCfg{0, 4, 4, 32, 4}, src, dst, A_R, omega);
  if ((g->jcfg.kind == 1 || g->jcfg.kind == 7) && g->maps_ready)
    return launch_jacobi_tma(L, g->jcfg, g->base + g->maps_off, src == A_P ? 0 : 1, dst,
                             omega);
  if (g->jcfg.kind == 2) return launch_jacobi_direct(L, g->jcfg, src, dst, A_R, omega);
  if (g->jcfg.kind == 3) return launch_jacobi_async(L, g->jcfg, src, dst, A_R, omega);

  return launch_jacobi(L, g->jcfg, src, dst, A_R, omega);
}

// iters sweeps of weight omega from 'start' (P or P2, ghosts current).
// With end == nullptr the result is copied into P if it lands in P2;
// otherwise *end receives the array holding it (ghosts current).
cfd_status enq_sweeps(cfd_grid* g, int iters, double omega, int start = A_P, int* end = nullptr) {
  const float om = (float)omega;
  int cur = start, oth = start == A_P ? A_P2 : A_P;
  cfd_status s;
  if (fused_ok(g)) {
    const Launch L = make_launch(g);
    // periodic two-sweep launches read two ghost layers of the iterate and
    // one of R, and write none: fill them before the first launch and the
    // output's after each
    const bool per = g->jcfg.kind == 9 && ws2_periodic(g);
    if (per && iters >= 2 && (s = enq_ghost(g, (1u << A_R) | (1u << cur))) != CFD_OK) return s;
    for (int it = 0; it + 1 < iters; it += 2) {
      if (g->jcfg.kind == 9)
        CK(g, launch_jacobi2_ws(L, g->jcfg, g->base + g->maps_off, cur == A_P ? 0 : 1, oth,
                                om, per));
      else
        CK(g, launch_jacobi2(L, g->jcfg, cur, oth, A_R, om));
      g->launches += 1;
      std::swap(cur, oth);
      if (per && (s = enq_ghost(g, 1u << cur)) != CFD_OK) return s;
    }
    if (iters % 2) {
      CK(g, sweep(g, L, cur, oth, om));
      g->launches += 1;
      std::swap(cur, oth);
    }
    iters = 0;
  }
  for (int it = 0; it < iters; ++it) {
    if ((s = each_launch(g, [&](const Launch& L) { return sweep(g, L, cur, oth, om); })) != CFD_OK)
      return s;
    std::swap(cur, oth);
  }
  if (end) {
    *end = cur;
    return CFD_OK;
  }
  if (cur != A_P) {
    const Launch L = make_launch(g);
    CK(g, launch_copy(L, g->scfg, cur, A_P));
    g->launches += 1;
  }
  return CFD_OK;
}

cfd_status enq_solve(cfd_grid* g, double c_dt, int iters) {
  cfd_status s = each_launch(g, [&](const Launch& L) {
    return launch_divergence(L, g->scfg, kSets[CFD_SET_W], (float)(1.0 / c_dt), A_R);
  });
  if (s != CFD_OK) return s;
  return enq_sweeps(g, iters, g->omega);
}

cfd_status enq_project(cfd_grid* g, double c_dt, int os, int p_arr = A_P) {
  cfd_status s = each_launch(g, [&](const Launch& L) {
    return launch_project(L, g->scfg, kSets[CFD_SET_W], p_arr, (float)c_dt, kSets[os]);
  });
  if (s != CFD_OK) return s;
  return enq_ghost(g, set_mask(os));
}

cfd_status enq_vcycle_p(cfd_grid* g);

// The pressure solve of a step's stage from the pressure in 'start' (P or
// P2): K Jacobi sweeps, or V-cycles; *end receives the array holding the
// result (the V-cycles keep it in P).
cfd_status enq_stage_solve(cfd_grid* g, double c_dt, int start, int* end) {
  if (g->solver != CFD_SOLVER_MG) {
    cfd_status s = enq_solve(g, c_dt, 0);
    return s != CFD_OK ? s : enq_sweeps(g, g->iters, g->omega, start, end);
  }
  if (start != A_P) {
    CK(g, launch_copy(make_launch(g), g->scfg, start, A_P));
    g->launches += 1;
  }
  cfd_status s = enq_solve(g, c_dt, 0);
  for (int c = 0; c < g->mg_cycles && s == CFD_OK; ++c) s = enq_vcycle_p(g);
  *end = A_P;
  return s;
}

// One projected Heun stage.  pcur: the array holding the pressure on entry,
// updated to the one holding it on exit (a step's second stage starts from
// where the first left it, so an odd number of ping-pong launches per solve
// needs no copy); with pcur == nullptr the pressure starts and ends in P.
cfd_status enq_rk_stage(cfd_grid* g, int stage, double dt, int* pcur = nullptr) {
  cfd_status s;
  int cur = pcur ? *pcur : A_P;
  const double cdt = stage == 1 ? dt : 0.5 * dt;
  if (stage == 1) {
    if ((s = enq_ghost(g, set_mask(CFD_SET_U) | (1u << cur))) != CFD_OK) return s;
    if ((s = enq_stage(g, 0.0, CFD_SET_U, 1.0, CFD_SET_U, dt, CFD_SET_W)) != CFD_OK) return s;
  } else {
    if ((s = enq_stage(g, 0.5, CFD_SET_U, 0.5, CFD_SET_U1, 0.5 * dt, CFD_SET_W)) != CFD_OK)
      return s;
  }
  // the stage output's ghosts: read only by the divergence (the normal
  // component below each low face), which takes a wall's value itself
  bool walls = true;
  for (int f = 0; f < 6; ++f) walls &= g->bc[f] == CFD_BC_WALL;
  if (!walls && (s = enq_ghost(g, set_mask(CFD_SET_W))) != CFD_OK) return s;
  if ((s = enq_stage_solve(g, cdt, cur, &cur)) != CFD_OK) return s;
  if ((s = enq_project(g, cdt, stage == 1 ? CFD_SET_U1 : CFD_SET_U, cur)) != CFD_OK) return s;
  if (pcur) {
    *pcur = cur;
  } else if (cur != A_P) {
    CK(g, launch_copy(make_launch(g), g->scfg, cur, A_P));
    g->launches += 1;
  }
  return CFD_OK;
}

// ------------------------------------------------------------- multigrid

int mg_depth(const cfd_grid* g) {
  const int avail = (int)g->mgl.size();
  return g->mg_levels > 0 ? std::min(g->mg_levels, avail) : avail;
}

cfd_status mg_supported(cfd_grid* g) {
  if (g->nblocks != 1 || g->dtype != CFD_F32)
    return fail(CFD_EUNSUPPORTED, "multigrid needs a single FP32 block");
  if (g->mgl.empty())
    return fail(CFD_EUNSUPPORTED, "multigrid needs every dimension even and >= 4");
  return CFD_OK;
}

// Launch over level l (0: the grid itself): one block, cell size 2^l h.
Launch level_launch(cfd_grid* g, int l) {
  Launch L = make_launch(g);
  if (l == 0) return L;
  L.blocks = reinterpret_cast<const BlockDev*>(g->base + g->mg_table_off) + (l - 1);
  L.b0 = 0;
  L.nblocks = 1;
  for (int d = 0; d < 3; ++d) {
    const double h = std::ldexp(g->h[d], l);
    L.ih[d] = (float)(1.0 / h);
    L.ih2[d] = (float)(1.0 / (h * h));
  }
  L.hn = reinterpret_cast<const int(*)[3]>(g->mg_hn.data() + 3 * (l - 1));
  return L;
}

MgView mg_view(cfd_grid* g, int l, int arr) {
  const BlockDev& d = l == 0 ? g->bdev[0] : g->mg_bdev[l - 1];
  MgView v;
  v.o = reinterpret_cast<float*>(g->base) + d.org[arr];
  for (int a = 0; a < 3; ++a) v.n[a] = d.n[a];
  v.py = d.py;
  v.pz = d.pz;
  return v;
}

// n weighted Jacobi sweeps on level l for L P = R from the array 'start'
// (P or P2); *end receives the array holding the result.  Coarse levels use
// the register sweep with a z chunk small enough to give every SM a few
// tiles (they are latency-bound, not bandwidth-bound).
cfd_status enq_level_sweeps(cfd_grid* g, int l, int n, int start, int* end) {
  if (l == 0) return enq_sweeps(g, n, g->mg_omega, start, end);
  const Launch L = level_launch(g, l);
  const int* dn = g->mg_hn.data() + 3 * (l - 1);
  const long long txy = (long long)((dn[0] + 127) / 128) * ((dn[1] + 3) / 4);
  const int zc = (int)std::max(1LL, std::min(32LL, dn[2] * txy / (4LL * g->sms)));
  int cur = start, oth = start == A_P ? A_P2 : A_P;
  for (int it = 0; it < n; ++it) {
    CK(g, launch_jacobi(L, JacobiCfg{0, 4, 4, zc, 4}, cur, oth, A_R, (float)g->mg_omega));
    g->launches += 1;
    std::swap(cur, oth);
  }
  *end = cur;
  return CFD_OK;
}

// Every ghost cell of level l's array arr (the prolongation reads edges and
// corners).
cfd_status enq_level_ghost(cfd_grid* g, int l, int arr) {
  if (l == 0) return enq_ghost(g, 1u << arr);
  const GhostItem* items = reinterpret_cast<const GhostItem*>(g->base + g->items_off) + g->gitem_first[l];
  CK(g, launch_ghost(level_launch(g, l), &arr, 1, items, g->gitem_count[l]));
  g->launches += 1;
  return CFD_OK;
}

// First level (>= 1) small enough for the one-CTA bottom of the cycle.
int mg_bottom_level(const cfd_grid* g, int depth) {
  for (int l = 1; l <= depth; ++l) {
    const int* n = g->mg_hn.data() + 3 * (l - 1);
    if ((long long)n[0] * n[1] * n[2] <= kMgBottomCells) return l;
  }
  return depth + 1;  // none
}

MgBottom mg_bottom_args(cfd_grid* g, int lb, int depth) {
  MgBottom b;
  memset(&b, 0, sizeof b);
  b.levels = depth - lb + 1;
  for (int q = 0; q < b.levels; ++q) {
    const Launch L = level_launch(g, lb + q);
    for (int a = 0; a < 3; ++a) {
      b.n[q][a] = g->mg_hn[3 * (lb + q - 1) + a];
      b.c[q][a] = L.ih2[a];
    }
    b.inv_diag[q] = 1.f / (2.f * (L.ih2[0] + L.ih2[1] + L.ih2[2]));
  }
  for (int a = 0; a < 3; ++a) b.per[a] = g->bc[2 * a] == CFD_BC_PERIODIC;
  b.nu1 = g->mg_nu1;
  b.nu2 = g->mg_nu2;
  b.ncoarse = g->mg_ncoarse;
  b.omega = (float)g->mg_omega;
  b.r_in = mg_view(g, lb, A_R);
  b.p_out = mg_view(g, lb, A_P);
  return b;
}

// One V-cycle from level l down to level depth (correction scheme).  *cur:
// the array (P or P2) holding level l's iterate, on entry and on exit.
cfd_status enq_vcycle(cfd_grid* g, int l, int depth, int* cur) {
  cfd_status s;
  if (l == depth) return enq_level_sweeps(g, l, g->mg_ncoarse, *cur, cur);
  if ((s = enq_level_sweeps(g, l, g->mg_nu1, *cur, cur)) != CFD_OK) return s;
  const Launch L = level_launch(g, l);
  CK(g, launch_mg_restrict(g->own, mg_view(g, l, *cur), mg_view(g, l, A_R).o,
                           mg_view(g, l + 1, A_R), L.ih2));
  g->launches += 1;
  int ccur = A_P;
  if (l + 1 == mg_bottom_level(g, depth)) {
    // levels l + 1 .. depth in one CTA; it writes level l + 1's P and ghosts
    CK(g, launch_mg_bottom(g->own, mg_bottom_args(g, l + 1, depth)));
    g->launches += 1;
  } else {
    const auto& c = g->mgl[l];
    CK(g, cudaMemsetAsync(g->base + c.first_byte, 0, c.array_bytes, g->own));  // zero correction
    if ((s = enq_vcycle(g, l + 1, depth, &ccur)) != CFD_OK) return s;
    if ((s = enq_level_ghost(g, l + 1, ccur)) != CFD_OK) return s;
  }
  const int per[3] = {g->bc[0] == CFD_BC_PERIODIC, g->bc[2] == CFD_BC_PERIODIC,
                      g->bc[4] == CFD_BC_PERIODIC};
  CK(g, launch_mg_prolong(g->own, mg_view(g, l, *cur), mg_view(g, l + 1, ccur), per));
  g->launches += 1;
  return enq_level_sweeps(g, l, g->mg_nu2, *cur, cur);
}

// One V-cycle on the grid's P (result in P).
cfd_status enq_vcycle_p(cfd_grid* g) {
  int cur = A_P;
  cfd_status s = enq_vcycle(g, 0, mg_depth(g), &cur);
  if (s != CFD_OK || cur == A_P) return s;
  CK(g, launch_copy(make_launch(g), g->scfg, cur, A_P));
  g->launches += 1;
  return CFD_OK;
}

// One V-cycle as a CUDA graph (captured once per configuration) and its
// replay: the coarse levels are many small launches.
cfd_status enq_vcycle_graph(cfd_grid* g) {
  if (!g->mg_valid) {
    if (g->mg_exec) {
      cudaGraphExecDestroy(g->mg_exec);
      g->mg_exec = nullptr;
    }
    CK(g, cudaStreamBeginCapture(g->own, cudaStreamCaptureModeThreadLocal));
    const long long before = g->launches;
    const cfd_status s = enq_vcycle_p(g);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(g->own, &graph);
    if (s != CFD_OK) {
      if (graph) cudaGraphDestroy(graph);
      return s;
    }
    if (e != cudaSuccess) return cuda_fail(g, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&g->mg_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(g, e, "cudaGraphInstantiate");
    g->mg_nodes = g->launches - before;
    g->launches = before;
    g->mg_valid = true;
  }
  CK(g, cudaGraphLaunch(g->mg_exec, g->own));
  g->launches += g->mg_nodes;
  return CFD_OK;
}

cfd_status run_reduce(cfd_grid* g, int mode, int set, double out[4]) {
  const Launch L = make_launch(g);
  double* partials = reinterpret_cast<double*>(g->base + g->partial_off);
  double* dout = reinterpret_cast<double*>(g->base + g->out_off);
  CK(g, launch_reduce(L, mode, mode == 0 ? kSets[set] : nullptr, A_P, A_R, partials, g->nparts, dout));
  g->launches += 2;
  CK(g, cudaMemcpyAsync(g->h_out, dout, 4 * sizeof(double), cudaMemcpyDeviceToHost, g->own));
  CK(g, cudaStreamSynchronize(g->own));
  for (int e = 0; e < 4; ++e) out[e] = g->h_out[e];
  return CFD_OK;
}

void invalidate_graph(cfd_grid* g) {
  g->graph_valid = false;
  g->mg_valid = false;
  drop_seg_graphs(g);
}

// ------------------------------------------------------------- adjoint

cfd_status adjoint_supported(cfd_grid* g) {
  if (g->nblocks != 1 || g->dtype != CFD_F32 || g->order != 2 || g->g < 2)
    return fail(CFD_EUNSUPPORTED,
                "the adjoint needs one FP32 block, order 2 and ghost width 2");
  if (g->solver != CFD_SOLVER_JACOBI)
    return fail(CFD_EUNSUPPORTED, "the adjoint transposes the Jacobi pressure solve only");
  for (int f = 0; f < 6; ++f)
    if (g->bc[f] != CFD_BC_PERIODIC) return fail(CFD_EUNSUPPORTED, "the adjoint needs periodic faces");
  return CFD_OK;
}

// Byte offset of element (-g,-g,-g) within an array's allocation, and of
// the interior origin.
size_t ghost_origin_bytes(const cfd_grid* g) { return (size_t)(kAlignBytes / g->es - g->g) * g->es; }
size_t interior_bytes(const cfd_grid* g) {
  const HostBlock& b = g->hb[0];
  return ((size_t)g->g * b.pz + (size_t)g->g * b.py + kAlignBytes / g->es) * g->es;
}
char* array_start(cfd_grid* g, int a) { return g->base + g->hb[0].first_byte + g->hb[0].array_bytes * a; }

cfd_status enq_adjoint_step(cfd_grid* g, double dt, const Ptr3& un, const Ptr3& u1, double* nu_acc) {
  const Launch L = make_launch(g);
  double diag = 0.0;
  for (int d = 0; d < 3; ++d) diag += 2.0 / (g->h[d] * g->h[d]);
  const float r_scale = (float)(-diag / g->omega);
  double* partials = reinterpret_cast<double*>(g->base + g->partial_off);
  const AdjSet lu{{A_LU, A_LV, A_LW}}, ws{{A_WU, A_WV, A_WW}}, u1s{{A_U1, A_V1, A_W1}};
  const unsigned m_lu = (1u << A_LU) | (1u << A_LV) | (1u << A_LW);
  cfd_status s;
  for (int stage = 2; stage >= 1; --stage) {
    const double c_dt = stage == 2 ? 0.5 * dt : dt;
    const AdjSet& lam_in = stage == 2 ? lu : u1s;
    if ((s = enq_ghost(g, stage == 2 ? m_lu : set_mask(CFD_SET_U1))) != CFD_OK) return s;
    CK(g, launch_adj_proj(L, lam_in, A_LP, (float)c_dt, r_scale, A_P, A_R));
    if ((s = enq_ghost(g, 1u << A_P)) != CFD_OK) return s;
    // the first K - 1 sweeps as a solve (two per launch where the variant
    // does that), the last one single, so that both of the last two
    // iterates are stored
    int cur = A_P, oth = A_P2;
    if (g->iters >= 2) {
      if ((s = enq_sweeps(g, g->iters - 1, g->omega, A_P, &cur)) != CFD_OK) return s;
      oth = cur == A_P ? A_P2 : A_P;
    }
    if (g->iters >= 1) {
      CK(g, sweep(g, L, cur, oth, (float)g->omega));
      g->launches += 1;
      std::swap(cur, oth);
    }
    // cur = b_{K+1}, oth = b_K (for K = 0, b_1 in both roles: lam_r = 0 path)
    CK(g, launch_adj_wp(L, lam_in, g->iters > 0 ? oth : cur, cur,
                        (float)(g->omega / diag / c_dt), ws, A_LP));
    if ((s = enq_ghost(g, set_mask(CFD_SET_W))) != CFD_OK) return s;
    if (stage == 2)
      CK(g, launch_adj_stage(L, ws, u1, u1s, 0, 0.5f, (float)(0.5 * dt), 1, lu, 0.5f, (float)g->nu,
                             partials, g->nparts, nu_acc, 0.5 * dt, g->form == CFD_FLUX));
    else
      CK(g, launch_adj_stage(L, ws, un, lu, 1, 1.0f, (float)dt, 0, lu, 0.0f, (float)g->nu,
                             partials, g->nparts, nu_acc, dt, g->form == CFD_FLUX));
    g->launches += 5;
  }
  return CFD_OK;
}

// ------------------------------------------------------------- autotuner
//
// Times candidate kernel variants on this grid (the Jacobi sweep, the RHS +
// stage kernel) and keeps the fastest.  Results are cached in a text file,
// one line per key "device|dtype|ghost|order|blocks": repeated runs on the
// same GPU model and grid reuse them without timing.

std::string tune_key(cfd_grid* g) {
  cudaDeviceProp prop;
  std::string name = "unknown";
  if (cudaGetDeviceProperties(&prop, g->device) == cudaSuccess) name = prop.name;
  for (auto& ch : name)
    if (ch == ' ' || ch == '|' || ch == '=') ch = '_';
  std::string dims;
  for (const auto& b : g->hb)
    dims += std::to_string(b.n[0]) + "x" + std::to_string(b.n[1]) + "x" + std::to_string(b.n[2]) + ",";
  unsigned long long hsh = 1469598103934665603ull;  // FNV-1a of the block dims
  for (char ch : dims) hsh = (hsh ^ (unsigned char)ch) * 1099511628211ull;
  char buf[160];
  snprintf(buf, sizeof buf, "%s|dt%d|g%d|o%d%s|nb%d|%016llx", name.c_str(), g->dtype, g->g, g->order,
           g->form == CFD_FLUX ? "f" : "", g->nblocks, hsh);
  return buf;
}

// Jacobi sweeps per timed region of the autotuner: the solve's count
// rounded down to a multiple of four, within 4 .. 16.
int tune_sweeps(const cfd_grid* g) { return std::min(16, std::max(4, g->iters / 4 * 4)); }

cfd_status time_region(cfd_grid* g, int reps, float* ms, int what) {
  cudaEvent_t a, b;
  CK(g, cudaEventCreate(&a));
  CK(g, cudaEventCreate(&b));
  CK(g, cudaEventRecord(a, g->own));
  cfd_status s = CFD_OK;
  for (int r = 0; r < reps && s == CFD_OK; ++r)
    // a multiple of four sweeps ends in P for every variant, so no copy is
    // timed, and as many as a solve takes up to 16, so that the ghost fill a
    // two-sweep solve makes before its first launch weighs as in a solve;
    // the RHS kernels are timed in both of a step's forms (stage 1 reads
    // one velocity set, stage 2 two)
    if (what == 0) {
      s = enq_sweeps(g, tune_sweeps(g), g->omega);
    } else {
      s = enq_stage(g, 0.0, CFD_SET_U, 1.0, CFD_SET_U, 1e-3, CFD_SET_W);
      if (s == CFD_OK) s = enq_stage(g, 0.5, CFD_SET_U, 0.5, CFD_SET_U1, 1e-3, CFD_SET_W);
    }
  CK(g, cudaEventRecord(b, g->own));
  CK(g, cudaEventSynchronize(b));
  CK(g, cudaEventElapsedTime(ms, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return s;
}

}  // namespace

namespace {
cfd_status ensure_step_graph(cfd_grid* g, double dt);
}  // namespace

// =================================================================== C ABI

extern "C" {

const char* cfd_last_error(void) { return t_err.c_str(); }

cfd_status cfd_grid_create(const int dims[3], int ghost, const double h[3], int storage,
                           void* stream, cfd_grid** out) {
  if (!dims || !out) return fail(CFD_EINVAL, "null argument");
  *out = nullptr;
  for (int d = 0; d < 3; ++d)
    if (dims[d] < 2 * ghost || dims[d] > (1 << 20))
      return fail(CFD_EINVAL, "dims[%d] = %d must be >= 2*ghost", d, dims[d]);
  cfd_grid* g = new cfd_grid();
  g->nblocks = 1;
  g->hb.resize(1);
  for (int d = 0; d < 3; ++d) {
    g->hb[0].n[d] = dims[d];
    g->hb[0].origin[d] = 0;
    g->gdims[d] = dims[d];
  }
  for (int f = 0; f < 6; ++f) g->hb[0].nbr[f] = 0;
  cfd_status s = common_init(g, ghost, h, storage, stream);
  if (s != CFD_OK) {
    destroy_handles(g);
    delete g;
    return s;
  }
  *out = g;
  return CFD_OK;
}

cfd_status cfd_blockset_create(int nblocks, const int* dims, const int* origin,
                               const int global_dims[3], int ghost, const double h[3],
                               int storage, void* stream, cfd_grid** out) {
  if (!dims || !origin || !global_dims || !out) return fail(CFD_EINVAL, "null argument");
  *out = nullptr;
  if (nblocks < 1 || nblocks > kMaxBlocks) return fail(CFD_EINVAL, "nblocks must be 1..%d", kMaxBlocks);
  // rectilinear tiling: per axis the distinct (origin, width) slabs partition [0, G)
  std::vector<std::pair<int, int>> slabs[3];
  for (int b = 0; b < nblocks; ++b)
    for (int d = 0; d < 3; ++d) {
      const int o = origin[3 * b + d], n = dims[3 * b + d];
      if (n < 2 * ghost) return fail(CFD_EINVAL, "block %d: dims[%d] = %d < 2*ghost", b, d, n);
      if (o < 0 || o + n > global_dims[d]) return fail(CFD_EINVAL, "block %d outside the domain", b);
      slabs[d].push_back({o, n});
    }
  for (int d = 0; d < 3; ++d) {
    std::sort(slabs[d].begin(), slabs[d].end());
    slabs[d].erase(std::unique(slabs[d].begin(), slabs[d].end()), slabs[d].end());
    int pos = 0;
    for (auto& s : slabs[d]) {
      if (s.first != pos) return fail(CFD_EINVAL, "axis %d: blocks do not form a rectilinear tiling", d);
      pos += s.second;
    }
    if (pos != global_dims[d]) return fail(CFD_EINVAL, "axis %d: slabs do not cover the domain", d);
  }
  const size_t ns[3] = {slabs[0].size(), slabs[1].size(), slabs[2].size()};
  if ((size_t)nblocks != ns[0] * ns[1] * ns[2])
    return fail(CFD_EINVAL, "blocks must be one per slab combination (%zu x %zu x %zu)", ns[0], ns[1], ns[2]);
  std::vector<int> at(nblocks, -1);
  std::vector<int> sidx(3 * nblocks);
  for (int b = 0; b < nblocks; ++b) {
    size_t lin = 0;
    for (int d = 2; d >= 0; --d) {
      const std::pair<int, int> key{origin[3 * b + d], dims[3 * b + d]};
      const size_t k = std::lower_bound(slabs[d].begin(), slabs[d].end(), key) - slabs[d].begin();
      sidx[3 * b + d] = (int)k;
      lin = lin * ns[d] + k;
    }
    if (at[lin] != -1) return fail(CFD_EINVAL, "blocks %d and %d coincide", at[lin], b);
    at[lin] = b;
  }
  cfd_grid* g = new cfd_grid();
  g->nblocks = nblocks;
  g->blockset = true;
  g->hb.resize(nblocks);
  for (int d = 0; d < 3; ++d) g->gdims[d] = global_dims[d];
  for (int b = 0; b < nblocks; ++b) {
    for (int d = 0; d < 3; ++d) {
      g->hb[b].n[d] = dims[3 * b + d];
      g->hb[b].origin[d] = origin[3 * b + d];
    }
    for (int d = 0; d < 3; ++d)
      for (int side = 0; side < 2; ++side) {
        int s3[3] = {sidx[3 * b], sidx[3 * b + 1], sidx[3 * b + 2]};
        s3[d] = (int)((s3[d] + (side ? 1 : (int)ns[d] - 1)) % ns[d]);
        const size_t lin = ((size_t)s3[2] * ns[1] + s3[1]) * ns[0] + s3[0];
        g->hb[b].nbr[2 * d + side] = at[lin];
      }
  }
  cfd_status s = common_init(g, ghost, h, storage, stream);
  if (s != CFD_OK) {
    destroy_handles(g);
    delete g;
    return s;
  }
  *out = g;
  return CFD_OK;
}

cfd_status cfd_grid_destroy(cfd_grid* g) {
  if (!g) return CFD_OK;
  destroy_handles(g);
  delete g;
  return CFD_OK;
}

cfd_status cfd_memory_bytes(const cfd_grid* g, size_t* bytes) {
  if (!g || !bytes) return fail(CFD_EINVAL, "null argument");
  *bytes = g->bytes;
  return CFD_OK;
}

cfd_status cfd_bind_memory(cfd_grid* g, void* dev_ptr, size_t bytes) {
  if (!g || !dev_ptr) return fail(CFD_EINVAL, "null argument");
  if (reinterpret_cast<uintptr_t>(dev_ptr) % 256) return fail(CFD_EINVAL, "memory must be 256-byte aligned");
  if (bytes < g->bytes) return fail(CFD_ENOMEM, "bound %zu bytes, need %zu", bytes, g->bytes);
  if (g->owns && g->base) cudaFree(g->base);
  g->owns = false;
  g->base = static_cast<char*>(dev_ptr);
  invalidate_graph(g);
  return upload_tables(g);
}

cfd_status cfd_alloc_memory(cfd_grid* g) {
  if (!g) return fail(CFD_EINVAL, "null grid");
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, g->bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(CFD_ENOMEM, "cudaMalloc(%zu): %s", g->bytes, cudaGetErrorString(e));
  }
  if (g->owns && g->base) cudaFree(g->base);
  g->base = static_cast<char*>(p);
  g->owns = true;
  invalidate_graph(g);
  return upload_tables(g);
}

cfd_status cfd_array_layout(const cfd_grid* g, int block, int array, long long* offset_bytes,
                            long long shape[3], long long strides[3], int* elem_bytes) {
  if (!g) return fail(CFD_EINVAL, "null grid");
  if (block < 0 || block >= g->nblocks) return fail(CFD_EINVAL, "block %d out of range", block);
  if (array < 0 || array >= kNumArrays) return fail(CFD_EINVAL, "array %d out of range", array);
  const HostBlock& b = g->hb[block];
  const int align_e = kAlignBytes / g->es;
  if (offset_bytes)
    *offset_bytes = (long long)(b.first_byte + b.array_bytes * array) + (long long)(align_e - g->g) * g->es;
  if (shape) {
    shape[0] = b.n[2] + 2 * g->g;
    shape[1] = b.n[1] + 2 * g->g;
    shape[2] = b.n[0] + 2 * g->g;
  }
  if (strides) {
    strides[0] = b.pz;
    strides[1] = b.py;
    strides[2] = 1;
  }
  if (elem_bytes) *elem_bytes = g->es;
  return CFD_OK;
}

cfd_status cfd_block_info(const cfd_grid* g, int block, int dims[3], int origin[3], int* ghost) {
  if (!g) return fail(CFD_EINVAL, "null grid");
  if (block < 0 || block >= g->nblocks) return fail(CFD_EINVAL, "block %d out of range", block);
  for (int d = 0; d < 3; ++d) {
    if (dims) dims[d] = g->hb[block].n[d];
    if (origin) origin[d] = g->hb[block].origin[d];
  }
  if (ghost) *ghost = g->g;
  return CFD_OK;
}

cfd_status cfd_set_bc(cfd_grid* g, int face, int kind, const double wall_velocity[3]) {
  if (!g) return fail(CFD_EINVAL, "null grid");
  if (face < 0 || face > 5) return fail(CFD_EINVAL, "face %d out of range 0..5", face);
  if (kind != CFD_BC_PERIODIC && kind != CFD_BC_WALL) return fail(CFD_EINVAL, "unknown bc kind %d", kind);
  if (kind == CFD_BC_WALL && g->blockset)
    return fail(CFD_EUNSUPPORTED, "walls are supported on single-block grids only");
  double v[3] = {0, 0, 0};
  if (wall_velocity)
    for (int c = 0; c < 3; ++c) v[c] = wall_velocity[c];
  if (kind == CFD_BC_WALL && v[face / 2] != 0.0)
    return fail(CFD_EINVAL, "wall velocity must be tangential (component %d is normal)", face / 2);
  g->bc[face] = kind;
  for (int c = 0; c < 3; ++c) g->wall[face][c] = kind == CFD_BC_WALL ? v[c] : 0.0;
  invalidate_graph(g);
  return upload_tables(g);
}

cfd_status cfd_set_params(cfd_grid* g, double nu, int jacobi_iters, double omega, int order) {
  if (!g) return fail(CFD_EINVAL, "null grid");
  if (!(nu >= 0.0) || !std::isfinite(nu)) return fail(CFD_EINVAL, "nu must be >= 0");
  if (jacobi_iters < 0) return fail(CFD_EINVAL, "jacobi_iters must be >= 0");
  if (!(omega > 0.0 && omega < 2.0)) return fail(CFD_EINVAL, "omega must be in (0, 2)");
  if (order != 2 && order != 4) return fail(CFD_EINVAL, "order must be 2 or 4");
  if (order == 4 && g->g < 2) return fail(CFD_EINVAL, "order 4 needs ghost width 2");
  if (order == 4 && g->form == CFD_FLUX) return fail(CFD_EINVAL, "the flux form is order 2");
  g->nu = nu;
  g->iters = jacobi_iters;
  g->omega = omega;
  g->order = order;
  invalidate_graph(g);
  return CFD_OK;
}

cfd_status cfd_set_advection(cfd_grid* g, int form) {
  if (!g) return fail(CFD_EINVAL, "null grid");
  if (form != CFD_ADVECTIVE && form != CFD_FLUX)
    return fail(CFD_EINVAL, "form must be CFD_ADVECTIVE or CFD_FLUX");
  if (form == CFD_FLUX && g->order != 2) return fail(CFD_EINVAL, "the flux form is order 2");
  g->form = form;
  invalidate_graph(g);
  return CFD_OK;
}

cfd_status cfd_ghost_fill(cfd_grid* g, unsigned mask) {
  const CallRange range("cfd_ghost_fill");
  cfd_status s = usable(g);
  if (s != CFD_OK) return s;
  if (mask >> kNumArrays) return fail(CFD_EINVAL, "mask has bits beyond the array ids");
  if ((s = join_in(g)) != CFD_OK) return s;
  if ((s = enq_ghost(g, mask)) != CFD_OK) return s;
  return join_out(g);
}

cfd_status cfd_stage(cfd_grid* g, double a, int x_set, double b, int y_set, double c, int out_set) {
  const CallRange range("cfd_stage");
  cfd_status s = usable(g);
  if (s != CFD_OK) return s;
  if (y_set < 0 || y_set > 2 || out_set < 0 || out_set > 2 || (a != 0.0 && (x_set < 0 || x_set > 2)))
    return fail(CFD_EINVAL, "velocity set ids are 0..2");
  if (out_set == y_set || (a != 0.0 && out_set == x_set))
    return fail(CFD_EINVAL, "output set must differ from the input sets");
  if ((s = join_in(g)) != CFD_OK) return s;
  if ((s = enq_stage(g, a, x_set, b, y_set, c, out_set)) != CFD_OK) return s;
  return join_out(g);
}

cfd_status cfd_rhs_eval(cfd_grid* g, void* const out_dev[3]) {
  const CallRange range("cfd_rhs_eval");
  if (out_dev && (!out_dev[0] || !out_dev[1] || !out_dev[2]))
    return fail(CFD_EINVAL, "out_dev must be NULL or hold three device pointers");
  cfd_status s = cfd_stage(g, 0.0, 0, 0.0, CFD_SET_U, 1.0, CFD_SET_W);
  if (s != CFD_OK || !out_dev) return s;
  if ((s = join_in(g)) != CFD_OK) return s;
  for (int c = 0; c < 3; ++c) {
    size_t off = 0;  // elements: the blocks' interiors one after the other
    for (int b = 0; b < g->nblocks; ++b) {
      Launch L = make_launch(g);
      L.b0 = b;
      L.nblocks = 1;
      CK(g, launch_pack(L, A_WU + c, static_cast<char*>(out_dev[c]) + off * g->es, 1));
      g->launches += 1;
      const HostBlock& hb = g->hb[b];
      off += (size_t)hb.n[0] * hb.n[1] * hb.n[2];
    }
  }
  return join_out(g);
}

cfd_status cfd_pressure_solve(cfd_grid* g, double c_dt, int iters, double* residual) {
  const CallRange range("cfd_pressure_solve");
  cfd_status s = usable(g);
  if (s != CFD_OK) return s;
  if (!(c_dt > 0.0) || iters < 0) return fail(CFD_EINVAL, "need c_dt > 0 and iters >= 0");
  if ((s = join_in(g)) != CFD_OK) return s;
  if ((s = enq_solve(g, c_dt, iters)) != CFD_OK) return s;
  if (residual) {
    double out[4];
    if ((s = run_reduce(g, 1, 0, out)) != CFD_OK) return s;
    *residual = std::sqrt(out[0]);
    if (out[3] != 0.0) return fail(CFD_ENONFINITE, "residual is not finite");
  }
  return join_out(g);
}

cfd_status cfd_pressure_solve_converged(cfd_grid* g, double c_dt, double rtol, int max_iters,
                                        int check_every, int* iters_done, double* residual) {
  const CallRange range("cfd_pressure_solve_converged");
  cfd_status s = usable(g);
  if (s != CFD_OK) return s;
  if (!(c_dt > 0.0) || !(rtol >= 0.0) || max_iters < 0 || check_every < 1)
    return fail(CFD_EINVAL, "need c_dt > 0, rtol >= 0, max_iters >= 0, check_every >= 1");
  if ((s = join_in(g)) != CFD_OK) return s;
  if ((s = enq_solve(g, c_dt, 0)) != CFD_OK) return s;  // R = (D W)/c_dt
  double out[4];
  if ((s = run_reduce(g, 2, 0, out)) != CFD_OK) return s;
  if (out[3] != 0.0) return fail(CFD_ENONFINITE, "right-hand side is not finite");
  const double target = rtol * std::sqrt(out[0]);
  int done = 0;
  double res = 0.0;
  if ((s = run_reduce(g, 1, 0, out)) != CFD_OK) return s;
  res = std::sqrt(out[0]);
  while (!(res <= target) && done < max_iters) {
    const int n = std::min(check_every, max_iters - done);
    if ((s = enq_sweeps(g, n, g->omega)) != CFD_OK) return s;
    done += n;
    if ((s = run_reduce(g, 1, 0, out)) != CFD_OK) return s;
    res = std::sqrt(out[0]);
    if (out[3] != 0.0) return fail(CFD_ENONFINITE, "residual is not finite");
  }
  if (iters_done) *iters_done = done;
  if (residual) *residual = res;
  return join_out(g);
}

cfd_status cfd_multigrid_levels(const cfd_grid* g, int* levels) {
  if (!g || !levels) return fail(CFD_EINVAL, "null argument");
  *levels = (int)g->mgl.size();
  return CFD_OK;
}

cfd_status cfd_set_multigrid(cfd_grid* g, int levels, int nu1, int nu2, int ncoarse,
                             double omega) {
  if (!g) return fail(CFD_EINVAL, "null grid");
  if (levels < 0 || nu1 < 0 || nu2 < 0 || ncoarse < 1 || !(omega > 0.0 && omega < 2.0))
    return fail(CFD_EINVAL, "need levels >= 0, nu1, nu2 >= 0, ncoarse >= 1, omega in (0, 2)");
  if (levels > (int)g->mgl.size())
    return fail(CFD_EINVAL, "only %d coarse levels are available", (int)g->mgl.size());
  g->mg_levels = levels;
  g->mg_nu1 = nu1;
  g->mg_nu2 = nu2;
  g->mg_ncoarse = ncoarse;
  g->mg_omega = omega;
  invalidate_graph(g);
  return CFD_OK;
}

cfd_status cfd_set_pressure_solver(cfd_grid* g, int solver, int cycles) {
  if (!g) return fail(CFD_EINVAL, "null grid");
  if (solver != CFD_SOLVER_JACOBI && solver != CFD_SOLVER_MG)
    return fail(CFD_EINVAL, "solver must be CFD_SOLVER_JACOBI or CFD_SOLVER_MG");
  if (solver == CFD_SOLVER_MG) {
    cfd_status s = mg_supported(g);
    if (s != CFD_OK) return s;
    if (cycles < 1) return fail(CFD_EINVAL, "cycles must be >= 1");
    g->mg_cycles = cycles;
  }
  g->solver = solver;
  invalidate_graph(g);
  return CFD_OK;
}

cfd_status cfd_mg_vcycles(cfd_grid* g, int cycles) {
  const CallRange range("cfd_mg_vcycles");
  cfd_status s = usable(g);
  if (s != CFD_OK) return s;
  if ((s = mg_supported(g)) != CFD_OK) return s;
  if (cycles < 0) return fail(CFD_EINVAL, "cycles must be >= 0");
  if ((s = join_in(g)) != CFD_OK) return s;
  for (int c = 0; c < cycles; ++c)
    if ((s = enq_vcycle_graph(g)) != CFD_OK) return s;
  return join_out(g);
}

cfd_status cfd_pressure_solve_mg(cfd_grid* g, double c_dt, double rtol, int max_cycles,
                                 int* cycles_done, double* residual) {
  const CallRange range("cfd_pressure_solve_mg");
  cfd_status s = usable(g);
  if (s != CFD_OK) return s;
  if ((s = mg_supported(g)) != CFD_OK) return s;
  if (!(c_dt > 0.0) || !(rtol >= 0.0) || max_cycles < 0)
    return fail(CFD_EINVAL, "need c_dt > 0, rtol >= 0, max_cycles >= 0");
  if ((s = join_in(g)) != CFD_OK) return s;
  if ((s = enq_solve(g, c_dt, 0)) != CFD_OK) return s;  // R = (D W)/c_dt
  double out[4];
  if ((s = run_reduce(g, 2, 0, out)) != CFD_OK) return s;
  if (out[3] != 0.0) return fail(CFD_ENONFINITE, "right-hand side is not finite");
  const double target = rtol * std::sqrt(out[0]);
  if ((s = run_reduce(g, 1, 0, out)) != CFD_OK) return s;
  double res = std::sqrt(out[0]);
  int done = 0;
  while (!(res <= target) && done < max_cycles) {
    if ((s = enq_vcycle_graph(g)) != CFD_OK) return s;
    ++done;
    if ((s = run_reduce(g, 1, 0, out)) != CFD_OK) return s;
    res = std::sqrt(out[0]);
    if (out[3] != 0.0) return fail(CFD_ENONFINITE, "residual is not finite");
  }
  if (cycles_done) *cycles_done = done;
  if (residual) *residual = res;
  return join_out(g);
}

cfd_status cfd_jacobi(cfd_grid* g, int iters) {
  const CallRange range("cfd_jacobi");
  cfd_status s = usable(g);
  if (s != CFD_OK) return s;
  if (iters < 0) return fail(CFD_EINVAL, "iters must be >= 0");
  if ((s = join_in(g)) != CFD_OK) return s;
  if ((s = enq_sweeps(g, iters, g->omega)) != CFD_OK) return s;
  return join_out(g);
}

cfd_status cfd_set_kernel_config(cfd_grid* g, const int jacobi[5], const int stencil[3]) {
  if (!g) return fail(CFD_EINVAL, "null grid");
  if (jacobi) {
    const JacobiCfg c{jacobi[0], jacobi[1], jacobi[2], jacobi[3], jacobi[4]};
    const bool ok0 = c.kind == 0 && (c.vx == 1 || c.vx == 2 || c.vx == 4) &&
                     (c.ty == 4 || c.ty == 8 || (c.ty == 16 && c.vx == 4));
    const bool ok1 = c.kind == 1 && ((c.vx == 4 && (c.ty == 4 || c.ty == 8 || c.ty == 16) &&
                                      (c.stages == 4 || c.stages == 6)) ||
                                     (c.vx == 2 && (c.ty == 8 || c.ty == 16) && c.stages == 4));
    const bool ok2 = c.kind == 2 && ((c.vx == 4 && ((c.ty == 4 && (c.zc == 1 || c.zc == 2 || c.zc == 4)) ||
                                                      (c.ty == 8 && c.zc == 1) || (c.ty == 2 && c.zc == 4))) ||
                                     (c.vx == 2 && c.ty == 4 && c.zc == 2) ||
                                     (c.vx == 1 && c.ty == 8 && c.zc == 1));
    const bool ok3 = c.kind == 3 && c.vx == (g->dtype == CFD_F32 ? 4 : 8) &&
                     (((c.ty == 4 || c.ty == 8) && (c.stages == 5 || c.stages == 6)) ||
                      (c.ty == 2 && c.stages == 6));
    const bool ok5 = c.kind == 5 && (c.ty == 4 || c.ty == 8);
    const bool ok7 = c.kind == 7 &&
                     ((c.vx == 4 && (c.ty == 4 || c.ty == 8 || c.ty == 16) &&
                       (c.stages == 6 || c.stages == 8)) ||
                      (c.vx == 2 && (c.ty == 8 || c.ty == 16) && c.stages == 6));
    const bool ok9 = c.kind == 9 &&
                     ((c.vx == 4 && ((c.ty == 16 && (c.stages == 6 || c.stages == 7)) ||
                                     (c.ty == 8 && (c.stages == 5 || c.stages == 6)))) ||
                      (c.vx == 2 && (c.ty == 16 || c.ty == 8) && c.stages == 6));
    if (!(ok0 || ok1 || ok2 || ok3 || ok5 || ok7 || ok9) || c.zc < 1)
      return fail(CFD_EINVAL, "unsupported Jacobi config");
    g->jcfg = c;
    cfd_status s = refresh_maps(g);
    if (s != CFD_OK) {
      g->jcfg.kind = 0;
      return s;
    }
  }
  if (stencil) {
    if ((stencil[0] != 4 && stencil[0] != 8) || stencil[1] < 1 ||
        (stencil[2] < 0 || stencil[2] > 4))
      return fail(CFD_EINVAL, "unsupported stencil config");
    g->scfg = StencilCfg{stencil[0], stencil[1], stencil[2]};
  }
  invalidate_graph(g);
  return CFD_OK;
}

cfd_status cfd_autotune(cfd_grid* g, const char* cache_path, double* sweep_us) {
  const CallRange range("cfd_autotune");
  cfd_status s = usable(g);
  if (s != CFD_OK) return s;
  const std::string key = tune_key(g);
  if (cache_path) {
    if (FILE* f = fopen(cache_path, "r")) {
      char line[512];
      while (fgets(line, sizeof line, f)) {
        char k[256];
        int j[5], st[3];
        double us = 0.0;
        if (sscanf(line, "key=%255s jacobi=%d,%d,%d,%d,%d stencil=%d,%d,%d sweep_us=%lf", k, &j[0],
                   &j[1], &j[2], &j[3], &j[4], &st[0], &st[1], &st[2], &us) == 10 && key == k) {
          fclose(f);
          if (sweep_us) *sweep_us = us;
          return cfd_set_kernel_config(g, j, st);
        }
      }
      fclose(f);
    }
  }
  if ((s = join_in(g)) != CFD_OK) return s;
  const Launch L = make_launch(g);
  CK(g, launch_copy(L, g->scfg, A_P, A_U1));  // keep the solver's warm start
  std::vector<JacobiCfg> cands;
  for (int zc : {16, 32, 64}) {
    for (int ty : {4, 8}) cands.push_back({0, 4, ty, zc, 4});
    cands.push_back({0, 4, 16, zc, 4});
    cands.push_back({0, 1, 8, zc, 4});
  }
  cands.push_back({0, 2, 8, 32, 4});
  for (int zc : {16, 32, 64, 128})
    for (int ty : {4, 8, 16})
      for (int st : {6, 8}) cands.push_back({7, 4, ty, zc, st});
  if (g->nblocks > 1)  // narrow blocks: 64-wide tiles waste fewer lanes
    for (int zc : {32, 64, 128})
      for (int ty : {8, 16}) cands.push_back({7, 2, ty, zc, 6});
  if (g->nblocks == 1)
    for (int zc : {16, 32, 64, 128})
      for (int ty : {4, 8}) cands.push_back({5, 4, ty, zc, 0});
  for (int zc : {32, 64})
    for (const JacobiCfg& d : {JacobiCfg{9, 4, 16, zc, 7}, JacobiCfg{9, 4, 16, zc, 6},
                               JacobiCfg{9, 4, 8, zc, 5}, JacobiCfg{9, 4, 8, zc, 6}})
      cands.push_back(d);
  if (g->nblocks > 1)  // two sweeps per launch on 64-wide tiles
    for (int zc : {16, 32, 64})
      for (int ty : {8, 16}) cands.push_back({9, 2, ty, zc, 6});
  const int avx = g->dtype == CFD_F32 ? 4 : 8;
  for (int zc : {16, 32, 64})
    for (const JacobiCfg& d : {JacobiCfg{3, avx, 4, zc, 5}, JacobiCfg{3, avx, 4, zc, 6},
                               JacobiCfg{3, avx, 8, zc, 5}, JacobiCfg{3, avx, 8, zc, 6},
                               JacobiCfg{3, avx, 2, zc, 6}})
      cands.push_back(d);
  for (const JacobiCfg& d : {JacobiCfg{2, 4, 4, 1, 0}, JacobiCfg{2, 4, 4, 2, 0}, JacobiCfg{2, 4, 8, 1, 0},
                             JacobiCfg{2, 4, 2, 4, 0}, JacobiCfg{2, 4, 4, 4, 0}, JacobiCfg{2, 2, 4, 2, 0},
                             JacobiCfg{2, 1, 8, 1, 0}})
    cands.push_back(d);
  for (int zc : {16, 32, 64}) {
    for (int ty : {4, 8, 16})
      for (int st : {4, 6}) cands.push_back({1, 4, ty, zc, st});
    cands.push_back({1, 2, 16, zc, 4});
  }
  const JacobiCfg saved = g->jcfg;
  JacobiCfg best = saved;
  float best_ms = 1e30f;
  for (const auto& c : cands) {
    g->jcfg = c;
    if (refresh_maps(g) != CFD_OK || ((c.kind == 1 || c.kind == 7 || c.kind == 9) && !g->maps_ready))
      continue;
    float ms = 0.f;
    if ((s = time_region(g, 1, &ms, 0)) != CFD_OK) return s;  // warm-up
    if ((s = time_region(g, 5, &ms, 0)) != CFD_OK) return s;
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  g->jcfg = best;
  if ((s = refresh_maps(g)) != CFD_OK) return s;
  CK(g, launch_copy(L, g->scfg, A_U1, A_P));
  StencilCfg sbest = g->scfg;
  float sbest_ms = 1e30f;
  const bool pair_ok = g->dtype == CFD_F32 && (g->order == 2 || g->form == CFD_FLUX);
  for (int tz : {0, 1, 2, 3, 4})
  for (int ty : {4, 8})
    for (int zc : {8, 16, 32, 64}) {
      if ((tz == 1 || tz == 3) && zc < 16) continue;
      if (tz == 3 && (ty != 4 || !pair_ok)) continue;  // the pair kernel's rows are fixed at 4
      g->scfg = StencilCfg{ty, zc, tz};
      float ms = 0.f;
      if ((s = time_region(g, 1, &ms, 1)) != CFD_OK) return s;
      if ((s = time_region(g, 3, &ms, 1)) != CFD_OK) return s;
      if (ms < sbest_ms) {
        sbest_ms = ms;
        sbest = g->scfg;
      }
    }
  g->scfg = sbest;
  invalidate_graph(g);
  const double us = best_ms * 1000.0 / (5.0 * tune_sweeps(g));  // 5 timed repetitions
  if (sweep_us) *sweep_us = us;
  if (cache_path) {
    if (FILE* f = fopen(cache_path, "a")) {
      fprintf(f, "key=%s jacobi=%d,%d,%d,%d,%d stencil=%d,%d,%d sweep_us=%.3f\n", key.c_str(),
              best.kind, best.vx, best.ty, best.zc, best.stages, sbest.ty, sbest.zc, sbest.tile_tz, us);
      fclose(f);
    }
  }
  return join_out(g);
}

cfd_status cfd_get_kernel_config(const cfd_grid* g, int jacobi[5], int stencil[3]) {
  if (!g) return fail(CFD_EINVAL, "null grid");
  if (jacobi) {
    jacobi[0] = (g->jcfg.kind == 1 || g->jcfg.kind == 7 || g->jcfg.kind == 9) && !g->maps_ready
                    ? 0
                    : g->jcfg.kind;
    jacobi[1] = g->jcfg.vx;
    jacobi[2] = g->jcfg.ty;
    jacobi[3] = g->jcfg.zc;
    jacobi[4] = g->jcfg.stages;
  }
  if (stencil) {
    stencil[0] = g->scfg.ty;
    stencil[1] = g->scfg.zc;
    stencil[2] = g->scfg.tile_tz;
  }
  return CFD_OK;
}

cfd_status cfd_set_launch_mode(cfd_grid* g, int per_block) {
  if (!g) return fail(CFD_EINVAL, "null grid");
  g->per_block = per_block != 0;
  invalidate_graph(g);
  return CFD_OK;
}

cfd_status cfd_stats(const cfd_grid* g, long long* kernel_launches) {
  if (!g || !kernel_launches) return fail(CFD_EINVAL, "null argument");
  *kernel_launches = g->launches;
  return CFD_OK;
}

cfd_status cfd_project(cfd_grid* g, double c_dt, int out_set) {
  const CallRange range("cfd_project");
  cfd_status s = usable(g);
  if (s != CFD_OK) return s;
  if (out_set < 0 || out_set > 2 || out_set == CFD_SET_W) return fail(CFD_EINVAL, "output set must be U or U1");
  if ((s = join_in(g)) != CFD_OK) return s;
  if ((s = enq_project(g, c_dt, out_set)) != CFD_OK) return s;
  return join_out(g);
}

cfd_status cfd_rk_step(cfd_grid* g, int stage, double dt) {
  const CallRange range("cfd_rk_step");
  cfd_status s = usable(g);
  if (s != CFD_OK) return s;
  if (stage != 1 && stage != 2) return fail(CFD_EINVAL, "stage must be 1 or 2");
  if (!(dt > 0.0)) return fail(CFD_EINVAL, "dt must be > 0");
  if ((s = join_in(g)) != CFD_OK) return s;
  if ((s = enq_rk_stage(g, stage, dt)) != CFD_OK) return s;
  if (stage == 2) {
    g->t += dt;
    g->step += 1;
  }
  return join_out(g);
}

cfd_status cfd_step(cfd_grid* g, double dt, int n) {
  const CallRange range("cfd_step");
  cfd_status s = usable(g);
  if (s != CFD_OK) return s;
  if (!(dt > 0.0) || n < 0) return fail(CFD_EINVAL, "need dt > 0 and n >= 0");
  if (n == 0) return CFD_OK;
  if ((s = join_in(g)) != CFD_OK) return s;
  if ((s = ensure_step_graph(g, dt)) != CFD_OK) return s;
  for (int i = 0; i < n; ++i) CK(g, cudaGraphLaunch(g->gexec, g->own));
  g->launches += n * g->graph_nodes;
  g->t += n * dt;
  g->step += n;
  return join_out(g);
}

cfd_status cfd_reduce(cfd_grid* g, int set, double* kinetic_energy, double* max_abs_u,
                      double* max_abs_div) {
  const CallRange range("cfd_reduce");
  cfd_status s = usable(g);
  if (s != CFD_OK) return s;
  if (set < 0 || set > 2) return fail(CFD_EINVAL, "set must be 0..2");
  if ((s = join_in(g)) != CFD_OK) return s;
  double out[4];
  if ((s = run_reduce(g, 0, set, out)) != CFD_OK) return s;
  if (kinetic_energy) *kinetic_energy = 0.5 * out[0] * g->h[0] * g->h[1] * g->h[2];
  if (max_abs_u) *max_abs_u = out[1];
  if (max_abs_div) *max_abs_div = out[2];
  if ((s = join_out(g)) != CFD_OK) return s;
  if (out[3] != 0.0) return fail(CFD_ENONFINITE, "%g non-finite velocity values", out[3]);
  return CFD_OK;
}

cfd_status cfd_residual(cfd_grid* g, double* residual) {
  const CallRange range("cfd_residual");
  cfd_status s = usable(g);
  if (s != CFD_OK) return s;
  if (!residual) return fail(CFD_EINVAL, "null argument");
  if ((s = join_in(g)) != CFD_OK) return s;
  double out[4];
  if ((s = run_reduce(g, 1, 0, out)) != CFD_OK) return s;
  *residual = std::sqrt(out[0]);
  if ((s = join_out(g)) != CFD_OK) return s;
  if (out[3] != 0.0) return fail(CFD_ENONFINITE, "residual is not finite");
  return CFD_OK;
}

cfd_status cfd_adjoint_step(cfd_grid* g, double dt, const void* const un[3],
                            const void* const u1[3], double* dnu_accum_dev) {
  const CallRange range("cfd_adjoint_step");
  cfd_status s = usable(g);
  if (s != CFD_OK) return s;
  if ((s = adjoint_supported(g)) != CFD_OK) return s;
  if (!un || !u1 || !dnu_accum_dev || !(dt > 0.0)) return fail(CFD_EINVAL, "bad argument");
  Ptr3 pn, p1;
  const size_t shift = interior_bytes(g) - ghost_origin_bytes(g);
  for (int c = 0; c < 3; ++c) {
    if (!un[c] || !u1[c]) return fail(CFD_EINVAL, "null state pointer");
    pn.p[c] = reinterpret_cast<const float*>(static_cast<const char*>(un[c]) + shift);
    p1.p[c] = reinterpret_cast<const float*>(static_cast<const char*>(u1[c]) + shift);
  }
  if ((s = join_in(g)) != CFD_OK) return s;
  if ((s = enq_adjoint_step(g, dt, pn, p1, dnu_accum_dev)) != CFD_OK) return s;
  return join_out(g);
}

cfd_status cfd_rollout_bytes(const cfd_grid* g, int nsteps, int seg, size_t* bytes) {
  if (!g || !bytes || nsteps < 1 || seg < 1) return fail(CFD_EINVAL, "bad argument");
  const size_t nck = (size_t)(nsteps + seg - 1) / seg;
  *bytes = g->hb[0].array_bytes * (4 * nck + 6 * (size_t)seg);
  return CFD_OK;
}

}  // extern "C"

namespace {

char* store_array(const cfd_grid* g, void* store, size_t slot) {
  return static_cast<char*>(store) + g->hb[0].array_bytes * slot;
}

cfd_status copy_arrays(cfd_grid* g, char* const* dst, char* const* src, int n) {
  for (int i = 0; i < n; ++i)
    CK(g, cudaMemcpyAsync(dst[i], src[i], g->hb[0].array_bytes, cudaMemcpyDeviceToDevice, g->own));
  return CFD_OK;
}

cfd_status ensure_step_graph(cfd_grid* g, double dt) {
  if (g->graph_valid && g->graph_dt == dt) return CFD_OK;
  if (g->gexec) {
    cudaGraphExecDestroy(g->gexec);
    g->gexec = nullptr;
  }
  CK(g, cudaStreamBeginCapture(g->own, cudaStreamCaptureModeThreadLocal));
  const long long before = g->launches;
  int pcur = A_P;  // the step leaves the pressure in P
  cfd_status s1 = enq_rk_stage(g, 1, dt, &pcur);
  cfd_status s2 = s1 == CFD_OK ? enq_rk_stage(g, 2, dt, &pcur) : s1;
  if (s2 == CFD_OK && pcur != A_P) {
    const cudaError_t ce = launch_copy(make_launch(g), g->scfg, pcur, A_P);
    g->launches += 1;
    if (ce != cudaSuccess) s2 = cuda_fail(g, ce, "launch_copy");
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(g->own, &graph);
  if (s2 != CFD_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s2;
  }
  if (e != cudaSuccess) return cuda_fail(g, e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&g->gexec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(g, e, "cudaGraphInstantiate");
  g->graph_valid = true;
  g->graph_dt = dt;
  g->graph_nodes = g->launches - before;
  g->launches = before;
  return CFD_OK;
}

// Recompute len steps from the current state, recording (u^n, u1) of step m
// in store slots; or the len adjoint steps in reverse.  Captured once per
// (store, dt, len) and replayed.
cfd_status seg_graph(cfd_grid* g, bool adjoint, int len, int seg, size_t nck, void* store,
                     double dt, cfd_grid::SegGraph** out) {
  if (g->seg_store != store || g->seg_dt != dt || g->seg_len != seg) {
    drop_seg_graphs(g);
    g->seg_store = store;
    g->seg_dt = dt;
    g->seg_len = seg;
  }
  cfd_grid::SegGraph* slots = adjoint ? g->adj_graph : g->rec_graph;
  for (int q = 0; q < 2; ++q)
    if (slots[q].exec && slots[q].len == len) {
      *out = &slots[q];
      return CFD_OK;
    }
  cfd_grid::SegGraph* tgt = slots[0].exec ? &slots[1] : &slots[0];
  if (tgt->exec) cudaGraphExecDestroy(tgt->exec);
  CK(g, cudaStreamBeginCapture(g->own, cudaStreamCaptureModeThreadLocal));
  const long long before = g->launches;
  cfd_status s = CFD_OK;
  double* nu_acc = reinterpret_cast<double*>(g->base + g->adj_off);
  const size_t shift = interior_bytes(g);
  for (int i = 0; i < len && s == CFD_OK; ++i) {
    const int m = adjoint ? len - 1 - i : i;
    char* rec[6];
    for (int c = 0; c < 6; ++c) rec[c] = store_array(g, store, 4 * nck + 6 * (size_t)m + c);
    if (!adjoint) {
      char* u[3] = {array_start(g, A_U), array_start(g, A_V), array_start(g, A_W)};
      char* u1[3] = {array_start(g, A_U1), array_start(g, A_V1), array_start(g, A_W1)};
      if ((s = copy_arrays(g, rec, u, 3)) != CFD_OK) break;
      if ((s = enq_rk_stage(g, 1, dt)) != CFD_OK) break;
      if ((s = copy_arrays(g, rec + 3, u1, 3)) != CFD_OK) break;
      s = enq_rk_stage(g, 2, dt);
    } else {
      Ptr3 pn, p1;
      for (int c = 0; c < 3; ++c) {
        pn.p[c] = reinterpret_cast<const float*>(rec[c] + shift);
        p1.p[c] = reinterpret_cast<const float*>(rec[3 + c] + shift);
      }
      s = enq_adjoint_step(g, dt, pn, p1, nu_acc);
    }
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(g->own, &graph);
  if (s != CFD_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  if (e != cudaSuccess) return cuda_fail(g, e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&tgt->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(g, e, "cudaGraphInstantiate");
  tgt->nodes = g->launches - before;
  tgt->len = len;
  g->launches = before;
  *out = tgt;
  return CFD_OK;
}

}  // namespace

extern "C" {

cfd_status cfd_rollout_forward(cfd_grid* g, double dt, int nsteps, int seg, void* store,
                               size_t bytes) {
  const CallRange range("cfd_rollout_forward");
  cfd_status s = usable(g);
  if (s != CFD_OK) return s;
  if ((s = adjoint_supported(g)) != CFD_OK) return s;
  size_t need = 0;
  if ((s = cfd_rollout_bytes(g, nsteps, seg, &need)) != CFD_OK) return s;
  if (!store || bytes < need || !(dt > 0.0)) return fail(CFD_EINVAL, "store too small or bad dt");
  if ((s = join_in(g)) != CFD_OK) return s;
  if ((s = ensure_step_graph(g, dt)) != CFD_OK) return s;
  char* st[4] = {array_start(g, A_U), array_start(g, A_V), array_start(g, A_W), array_start(g, A_P)};
  for (int n = 0; n < nsteps; ++n) {
    if (n % seg == 0) {
      char* ck[4];
      for (int c = 0; c < 4; ++c) ck[c] = store_array(g, store, 4 * (size_t)(n / seg) + c);
      if ((s = copy_arrays(g, ck, st, 4)) != CFD_OK) return s;
    }
    CK(g, cudaGraphLaunch(g->gexec, g->own));
    g->launches += g->graph_nodes;
  }
  g->t += nsteps * dt;
  g->step += nsteps;
  return join_out(g);
}

cfd_status cfd_rollout_backward(cfd_grid* g, double dt, int nsteps, int seg, void* store,
                                size_t bytes, double* dnu) {
  const CallRange range("cfd_rollout_backward");
  cfd_status s = usable(g);
  if (s != CFD_OK) return s;
  if ((s = adjoint_supported(g)) != CFD_OK) return s;
  size_t need = 0;
  if ((s = cfd_rollout_bytes(g, nsteps, seg, &need)) != CFD_OK) return s;
  if (!store || bytes < need || !(dt > 0.0)) return fail(CFD_EINVAL, "store too small or bad dt");
  const size_t nck = (size_t)(nsteps + seg - 1) / seg;
  if ((s = join_in(g)) != CFD_OK) return s;
  double* nu_acc = reinterpret_cast<double*>(g->base + g->adj_off);
  CK(g, cudaMemsetAsync(nu_acc, 0, sizeof(double), g->own));
  char* st[4] = {array_start(g, A_U), array_start(g, A_V), array_start(g, A_W), array_start(g, A_P)};
  for (long long sg = (long long)nck - 1; sg >= 0; --sg) {
    const int n0 = (int)sg * seg, len = std::min(seg, nsteps - n0);
    char* ck[4];
    for (int c = 0; c < 4; ++c) ck[c] = store_array(g, store, 4 * (size_t)sg + c);
    if ((s = copy_arrays(g, st, ck, 4)) != CFD_OK) return s;
    cfd_grid::SegGraph* rg = nullptr;
    if ((s = seg_graph(g, false, len, seg, nck, store, dt, &rg)) != CFD_OK) return s;
    CK(g, cudaGraphLaunch(rg->exec, g->own));
    g->launches += rg->nodes;
    cfd_grid::SegGraph* ag = nullptr;
    if ((s = seg_graph(g, true, len, seg, nck, store, dt, &ag)) != CFD_OK) return s;
    CK(g, cudaGraphLaunch(ag->exec, g->own));
    g->launches += ag->nodes;
  }
  CK(g, cudaMemcpyAsync(g->h_out, nu_acc, sizeof(double), cudaMemcpyDeviceToHost, g->own));
  CK(g, cudaStreamSynchronize(g->own));
  if (dnu) *dnu = g->h_out[0];
  return join_out(g);
}

cfd_status cfd_get_state(const cfd_grid* g, double* t, long long* step) {
  if (!g) return fail(CFD_EINVAL, "null grid");
  if (t) *t = g->t;
  if (step) *step = g->step;
  return CFD_OK;
}

cfd_status cfd_set_state(cfd_grid* g, double t, long long step) {
  if (!g) return fail(CFD_EINVAL, "null grid");
  g->t = t;
  g->step = step;
  return CFD_OK;
}

cfd_status cfd_copy_interior(cfd_grid* g, int block, int array, void* host, int to_device) {
  const CallRange range("cfd_copy_interior");
  cfd_status s = usable(g);
  if (s != CFD_OK) return s;
  if (!host) return fail(CFD_EINVAL, "null host pointer");
  if (block < 0 || block >= g->nblocks || array < 0 || array >= kNumArrays)
    return fail(CFD_EINVAL, "block or array id out of range");
  // Page-locked host memory is read or written by the pack kernel itself
  // over the host link (as fast as the copy engines here, and no second
  // pass); other host memory goes through one contiguous copy to or from
  // the staging region and the kernel between the staging region and the
  // padded array.
  const HostBlock& b = g->hb[block];
  const size_t bytes = (size_t)b.n[0] * b.n[1] * b.n[2] * g->es;
  Launch L = make_launch(g);
  L.b0 = block;
  L.nblocks = 1;
  cudaPointerAttributes pa{};
  void* direct = nullptr;
  if (cudaPointerGetAttributes(&pa, host) == cudaSuccess) {
    if (pa.type == cudaMemoryTypeHost && pa.devicePointer && g->host_copy != CFD_HOST_COPY_ENGINE)
      direct = pa.devicePointer;
  } else {
    cudaGetLastError();  // clear the query's error for plain host memory
  }
  if ((s = join_in(g)) != CFD_OK) return s;
  if (direct && g->host_copy == CFD_HOST_COPY_NARROW &&
      launch_pack_narrow(L, array, direct, to_device ? 0 : 1) == cudaSuccess) {
    // transferred by the narrow pack kernel
  } else if (direct) {
    CK(g, launch_pack(L, array, direct, to_device ? 0 : 1));
  } else {
    char* stage = g->base + g->staging_off;
    if (to_device) {
      CK(g, cudaMemcpyAsync(stage, host, bytes, cudaMemcpyDefault, g->own));
      CK(g, launch_pack(L, array, stage, 0));
    } else {
      CK(g, launch_pack(L, array, stage, 1));
      CK(g, cudaMemcpyAsync(host, stage, bytes, cudaMemcpyDefault, g->own));
    }
  }
  g->launches += 1;
  return join_out(g);
}

cfd_status cfd_set_host_copy(cfd_grid* g, int mode) {
  if (!g) return fail(CFD_EINVAL, "null grid");
  if (mode != CFD_HOST_COPY_KERNEL && mode != CFD_HOST_COPY_ENGINE && mode != CFD_HOST_COPY_NARROW)
    return fail(CFD_EINVAL,
                "mode must be CFD_HOST_COPY_KERNEL, CFD_HOST_COPY_ENGINE or CFD_HOST_COPY_NARROW");
  g->host_copy = mode;
  return CFD_OK;
}

cfd_status cfd_selftest_wait_timeout(cfd_grid* g, int form) {
  const CallRange range("cfd_selftest_wait_timeout");
  cfd_status s = usable(g);
  if (s != CFD_OK) return s;
  if (form != 0 && form != 1) return fail(CFD_EINVAL, "form must be 0 or 1");
  if ((s = join_in(g)) != CFD_OK) return s;
  CK(g, launch_wait_probe(make_launch(g), form));
  g->launches += 1;
  return join_out(g);
}

cfd_status cfd_check(cfd_grid* g) {
  const CallRange range("cfd_check");
  if (!g) return fail(CFD_EINVAL, "null grid");
  if (g->sticky) return fail(CFD_ECUDA, "grid is in a failed state after an earlier CUDA error");
  if (!g->base) return CFD_OK;
  CK(g, cudaMemcpyAsync(g->h_flag, g->base + g->flag_off, sizeof(int), cudaMemcpyDeviceToHost, g->own));
  CK(g, cudaStreamSynchronize(g->own));
  CK(g, cudaGetLastError());
  if (*g->h_flag != 0) return fail(CFD_ETIMEOUT, "device error flag %d", *g->h_flag);
  return CFD_OK;
}

}  // extern "C"
