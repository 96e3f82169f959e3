// libhfx C ABI: context, block registry, planning and the build driver.
//
// Build (Algorithm 5, "Calculate exact-exchange"):
//   1. pack the set blocks of each kind into one key-sorted device array and
//      take every block's upper limit max|x| (Sec. III.B);
//   2. plan: neighbour lists N[x] from the C keys, one work item per V block
//      <A,B> with A in the home cell (Algorithm 2/3 loop over <A,B>);
//   3. screen every (A,B,G) x F x variant with the block-norm product and
//      collect the Sigma key set (Sec. III.C, Algorithm 4 level 1);
//   4. contract the survivors in waves of work items sized to the scratch
//      budget (Algorithm 3, C((VC)D) order);
//   5. convert the fixed-point Sigma accumulators to FP64 and reduce E_X.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <memory>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "hfx_internal.h"
#include "hfx_split.h"

namespace {

template <class T>
struct DevBuf {
  T *p = nullptr;
  size_t n = 0;
  DevBuf() = default;
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  // grow-only; contents are not preserved
  cudaError_t reserve(size_t count) {
    if (count <= n && p) return cudaSuccess;
    release();
    const size_t c = count > 0 ? count : 1;
    cudaError_t e = cudaMalloc((void **)&p, c * sizeof(T));
    if (e != cudaSuccess) { p = nullptr; n = 0; return e; }
    n = c;
    return cudaSuccess;
  }
};

struct Entry {
  int32_t chunk;   // -1: host pending buffer
  int64_t off;
  int64_t len;
};

struct Chunk {
  double *dev = nullptr;
  size_t n = 0;
};

struct Kind {
  char name = '?';
  std::unordered_map<uint64_t, Entry> map;
  std::vector<Chunk> chunks;
  std::vector<double> pending;
  bool dirty = true;         // data or keys changed since the last pack
  bool keys_changed = true;  // key set changed since the last plan
  std::vector<uint64_t> keys;   // sorted, valid after pack
  std::vector<int64_t> offs;    // n + 1
  DevBuf<double> data;
  DevBuf<int64_t> d_offs;
  DevBuf<double> maxabs;
  bool data_is_chunk = false;   // data.p aliases chunks[0]

  ~Kind() { free_chunks(); }
  void free_chunks() {
    for (auto &c : chunks) {
      if (c.dev && !(data_is_chunk && c.dev == data.p)) cudaFree(c.dev);
    }
    chunks.clear();
  }
};

}  // namespace

// The merged system of the last hfx_build_batch whose first cell is this
// context, kept for the next batch of the same cells: identified by the
// cells' ids and the change counters of their C, V and D blocks.
struct BatchCache {
  std::vector<uint64_t> ids;
  std::vector<std::array<uint64_t, 3>> gens, kgens;
  std::vector<int32_t> first;
  hfx_ctx *merged = nullptr;
  ~BatchCache() { hfx_destroy(merged); }
};

static std::atomic<uint64_t> g_next_ctx_id{1};

struct hfx_ctx {
  uint64_t id = g_next_ctx_id.fetch_add(1);  // unique for the process
  uint64_t gen[3] = {0, 0, 0};               // changes of the C, V and D blocks
  uint64_t kgen[3] = {0, 0, 0};              // changes of their key sets
  std::unique_ptr<BatchCache> batch;
  int32_t natoms = 0;
  std::vector<int32_t> nao, nabf;
  double lattice[9] = {0};
  std::vector<double> pos;
  cudaStream_t stream = nullptr;
  Kind K[3];  // C, V, D
  std::string err;

  // plan (depends on the C and V key sets; dab on the D key set)
  bool plan_valid = false;
  std::vector<NbrEntry> nbr;
  std::vector<int64_t> nc_start;
  std::vector<int64_t> aotot;   // sum of nao over each atom's neighbour list
  std::vector<WorkItem> items;
  int64_t nwg = 0, nwf = 0, nmask = 0;
  DevBuf<NbrEntry> d_nbr;
  DevBuf<WorkItem> d_items;
  DevBuf<int32_t> d_nao, d_nabf, d_ncol;
  std::unordered_map<uint64_t, int64_t> dindex;
  DevBuf<uint64_t> d_dhkeys;
  DevBuf<int64_t> d_dhvals;
  uint64_t dmask = 0;

  // screen
  DevBuf<uint32_t> d_masks;
  DevBuf<uint8_t> d_wg;
  DevBuf<uint32_t> d_wf;
  DevBuf<unsigned long long> d_stab;
  uint64_t stab_cap = 0;
  DevBuf<unsigned long long> d_counters;
  DevBuf<unsigned> d_err;
  DevBuf<unsigned long long> d_collect;

  // Sigma
  std::vector<uint64_t> sig_keys;
  std::vector<int64_t> sig_offs;
  DevBuf<uint64_t> d_skeys;
  DevBuf<int64_t> d_soffs;
  DevBuf<uint64_t> d_shkeys;
  DevBuf<int64_t> d_shvals;
  uint64_t smask = 0;
  DevBuf<unsigned long long> d_acc;
  DevBuf<double> d_sigma;
  DevBuf<double> d_partials;
  DevBuf<double> d_ex;

  // scratch
  DevBuf<double> d_scratch;
  DevBuf<int64_t> d_waveoffs;

  // split-precision (HFX_OZAKI) operands
  int split_ks = 0;
  DevBuf<__nv_bfloat16> d_cy, d_c4, d_vs, d_ps, d_cz;
  DevBuf<int16_t> d_cy_e, d_c4_e, d_vs_e, d_ps_e, d_cz_e;
  DevBuf<int64_t> d_cz_meta;      // cz_base, cz_rowpre
  DevBuf<int32_t> d_kofs, d_ktotZ;
  DevBuf<int16_t> d_colG;          // per (atom, column): index of its neighbour entry
  DevBuf<int64_t> d_coloff;        // per atom: first column in d_colG
  std::vector<int32_t> ktotZ_h;  // per atom: sum of 16 ceil(nao / 16) over its neighbours
  int64_t h_cz_rows = 0;
  // D digit tiles for the D_FG / D_FB products
  DevBuf<__nv_bfloat16> d_dz, d_dzero;
  DevBuf<int64_t> d_dz_off;
  DevBuf<int32_t> d_dij, d_aoff;
  DevBuf<unsigned long long> d_de;
  int64_t dz_nd = -1;           // D blocks the tile metadata was built for (-1: stale)
  int dz_ks = 0;
  int kbmax = 16;
  ZcPlanShape zc_shape{16, 16, 0};
  int nsm = 0;
  DevBuf<ZcJob> d_zcjobs;
  DevBuf<ZcEnt> d_zcents;
  DevBuf<int> d_zckeys;           // job-cost histogram / range starts (256)
  DevBuf<long long> d_ctans;      // per-CTA busy time of the last D_FG / D_FB launch
  DevBuf<int64_t> d_split_meta;   // cy_base, cy_rowpre, c4_base, c4_rowpre, vs_base, v_rowpre, nc_start
  DevBuf<int32_t> d_kt;           // ktY, kt4
  std::vector<int32_t> ktY, kt4;
  int64_t h_cy_rows = 0, h_c4_rows = 0, h_v_rows = 0;
  DevBuf<int64_t> d_wave_split;   // p_rowpre, ps_base, y_candpre, v4_candpre
  DevBuf<Job> d_jobs, d_jobs4;
  DevBuf<int> d_njobs;
  DevBuf<unsigned long long> d_tmacs;
  cudaEvent_t sev[4] = {nullptr, nullptr, nullptr, nullptr};

  // Cauchy-Schwarz ERI screen (off while eps_eri < 0); bounds per C block,
  // recomputed when C or V change
  double eps_eri = -1.0;
  bool eri_valid = false;
  DevBuf<double> d_eri_sq;

  // batch builds: per-atom screening threshold of the merged cells (empty:
  // the build's theta), and whether this context's results came from a batch
  std::vector<double> theta_atom;
  DevBuf<double> d_theta_atom;
  bool from_batch = false;
  DevBuf<double> d_ex_cells;

  bool sym = false;             // V and D blocks all have transposed mirrors
  std::vector<int32_t> owner;   // shard: central atom -> rank (empty: no shard)
  int32_t rank = 0;
  bool c_reordered = false;     // C values changed: neighbour order must be rebuilt
  bool results_valid = false;
  double ex = 0.0;
  hfx_stats_v1 stats{};
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t kev[10] = {nullptr};  // per-kernel marks
  int64_t launches = 0;
};

namespace {

hfx_status fail(hfx_ctx *c, hfx_status s, const std::string &msg) {
  if (c) c->err = msg;
  return s;
}
hfx_status fail_cuda(hfx_ctx *c, const char *what, cudaError_t e) {
  return fail(c, HFX_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                   \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return fail_cuda(ctx, #call, e_);       \
  } while (0)

int kind_index(char w) { return w == 'C' ? 0 : w == 'V' ? 1 : w == 'D' ? 2 : -1; }

int64_t block_len(const hfx_ctx *ctx, int k, int i, int j) {
  if (k == 0) return (int64_t)ctx->nabf[i] * ctx->nao[i] * ctx->nao[j];
  if (k == 1) return (int64_t)ctx->nabf[i] * ctx->nabf[j];
  return (int64_t)ctx->nao[i] * ctx->nao[j];
}

bool key_ok(const hfx_ctx *ctx, const int32_t *k) {
  if (k[0] < 0 || k[0] >= ctx->natoms || k[1] < 0 || k[1] >= ctx->natoms) return false;
  for (int d = 2; d < 5; ++d)
    if (k[d] < -127 || k[d] > 127) return false;
  return true;
}

void invalidate(hfx_ctx *ctx, int k, bool keys) {
  ctx->K[k].dirty = true;
  ++ctx->gen[k];
  if (keys) ++ctx->kgen[k];
  if (k < 2) ctx->eri_valid = false;
  if (keys) ctx->K[k].keys_changed = true;
  if (keys && k == 2) ctx->dz_nd = -1;
  ctx->results_valid = false;
}

uint64_t pow2_at_least(uint64_t x) {
  uint64_t c = 16;
  while (c < x) c <<= 1;
  return c;
}

// Host-built open-addressing table (same probe sequence as dh_find).
void build_table(const std::vector<uint64_t> &keys, const std::vector<int64_t> &vals,
                 std::vector<uint64_t> &tk, std::vector<int64_t> &tv, uint64_t &mask) {
  const uint64_t cap = pow2_at_least(2 * keys.size() + 16);
  tk.assign(cap, HK_EMPTY);
  tv.assign(cap, -1);
  mask = cap - 1;
  for (size_t e = 0; e < keys.size(); ++e) {
    uint64_t s = hk_mix(keys[e]) & mask;
    while (tk[s] != HK_EMPTY) s = (s + 1) & mask;
    tk[s] = keys[e];
    tv[s] = vals[e];
  }
}

// Pack one kind into a key-sorted device array and compute block upper limits.
hfx_status pack_kind(hfx_ctx *ctx, int k) {
  Kind &K = ctx->K[k];
  if (!K.dirty) return HFX_OK;
  cudaStream_t st = ctx->stream;
  // flush host-side single-block sets
  if (!K.pending.empty()) {
    Chunk c;
    c.n = K.pending.size();
    CK(cudaMalloc((void **)&c.dev, c.n * sizeof(double)));
    CK(cudaMemcpyAsync(c.dev, K.pending.data(), c.n * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    const int32_t id = (int32_t)K.chunks.size();
    K.chunks.push_back(c);
    for (auto &kv : K.map)
      if (kv.second.chunk < 0) kv.second.chunk = id;
    K.pending.clear();
    K.pending.shrink_to_fit();
  }
  // free chunks no block refers to any more (every block they held was set
  // again), so that a full re-set of a kind leaves one chunk to adopt
  {
    std::vector<char> used(K.chunks.size(), 0);
    for (auto &kv : K.map)
      if (kv.second.chunk >= 0) used[kv.second.chunk] = 1;
    std::vector<int32_t> remap(K.chunks.size(), -1);
    std::vector<Chunk> keep;
    for (size_t c = 0; c < K.chunks.size(); ++c) {
      if (used[c]) {
        remap[c] = (int32_t)keep.size();
        keep.push_back(K.chunks[c]);
        continue;
      }
      if (K.data_is_chunk && K.chunks[c].dev == K.data.p) {
        K.data.p = nullptr;
        K.data.n = 0;
        K.data_is_chunk = false;
      }
      if (K.chunks[c].dev) cudaFree(K.chunks[c].dev);
    }
    if (keep.size() != K.chunks.size()) {
      K.chunks.swap(keep);
      for (auto &kv : K.map)
        if (kv.second.chunk >= 0) kv.second.chunk = remap[kv.second.chunk];
    }
  }
  const int64_t nblk = (int64_t)K.map.size();
  K.keys.clear();
  K.keys.reserve(nblk);
  for (auto &kv : K.map) K.keys.push_back(kv.first);
  std::sort(K.keys.begin(), K.keys.end());
  K.offs.assign(nblk + 1, 0);
  for (int64_t e = 0; e < nblk; ++e) K.offs[e + 1] = K.offs[e] + K.map[K.keys[e]].len;
  const int64_t total = K.offs[nblk];
  // fast path: one chunk that already holds exactly this packing
  bool adopt = K.chunks.size() == 1 && K.chunks[0].n == (size_t)total;
  for (int64_t e = 0; adopt && e < nblk; ++e) {
    const Entry &en = K.map[K.keys[e]];
    adopt = en.chunk == 0 && en.off == K.offs[e];
  }
  if (adopt) {
    if (!K.data_is_chunk) K.data.release();
    K.data.p = K.chunks[0].dev;
    K.data.n = K.chunks[0].n;
    K.data_is_chunk = true;
  } else {
    double *dst = nullptr;
    CK(cudaMalloc((void **)&dst, (size_t)(total > 0 ? total : 1) * sizeof(double)));
    std::vector<const double *> src(nblk);
    std::vector<int64_t> doff(nblk), len(nblk);
    for (int64_t e = 0; e < nblk; ++e) {
      const Entry &en = K.map[K.keys[e]];
      const double *base = en.chunk >= 0 ? K.chunks[en.chunk].dev
                                         : (K.data_is_chunk ? K.data.p : K.data.p);
      src[e] = base + en.off;
      doff[e] = K.offs[e];
      len[e] = en.len;
    }
    const double **d_src = nullptr;
    int64_t *d_doff = nullptr, *d_len = nullptr;
    CK(cudaMalloc((void **)&d_src, sizeof(double *) * (nblk > 0 ? nblk : 1)));
    CK(cudaMalloc((void **)&d_doff, sizeof(int64_t) * (nblk > 0 ? nblk : 1)));
    CK(cudaMalloc((void **)&d_len, sizeof(int64_t) * (nblk > 0 ? nblk : 1)));
    CK(cudaMemcpyAsync(d_src, src.data(), sizeof(double *) * nblk, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_doff, doff.data(), sizeof(int64_t) * nblk, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_len, len.data(), sizeof(int64_t) * nblk, cudaMemcpyHostToDevice, st));
    CK(launch_gather(d_src, d_doff, d_len, nblk, dst, st));
    ctx->launches += nblk > 0;
    CK(cudaStreamSynchronize(st));
    cudaFree(d_src);
    cudaFree(d_doff);
    cudaFree(d_len);
    // the packed array becomes the only chunk
    double *old_data = K.data_is_chunk ? nullptr : K.data.p;
    K.data.p = nullptr;
    K.data.n = 0;
    if (old_data) cudaFree(old_data);
    K.data_is_chunk = false;
    K.free_chunks();
    Chunk c;
    c.dev = dst;
    c.n = (size_t)total;
    K.chunks.push_back(c);
    K.data.p = dst;
    K.data.n = (size_t)total;
    K.data_is_chunk = true;
  }
  for (int64_t e = 0; e < nblk; ++e) {
    Entry &en = K.map[K.keys[e]];
    en.chunk = 0;
    en.off = K.offs[e];
  }
  CK(K.d_offs.reserve(nblk + 1));
  CK(cudaMemcpyAsync(K.d_offs.p, K.offs.data(), sizeof(int64_t) * (nblk + 1),
                     cudaMemcpyHostToDevice, st));
  CK(K.maxabs.reserve(nblk));
  CK(launch_maxabs(K.data.p, K.d_offs.p, nblk, K.maxabs.p, ctx->d_err.p, st));
  ctx->launches += nblk > 0;
  K.dirty = false;
  return HFX_OK;
}

// Neighbour lists and work items from the C and V key sets; D lookups.
hfx_status build_plan(hfx_ctx *ctx) {
  Kind &C = ctx->K[0], &V = ctx->K[1], &D = ctx->K[2];
  cudaStream_t st = ctx->stream;
  const bool cv_changed = C.keys_changed || V.keys_changed || !ctx->plan_valid || ctx->c_reordered;
  if (cv_changed) {
    const int n = ctx->natoms;
    ctx->nc_start.assign(n + 1, 0);
    ctx->nbr.resize(C.keys.size());
    for (size_t e = 0; e < C.keys.size(); ++e) {
      int32_t k[5];
      hk_unpack(C.keys[e], k);
      ctx->nc_start[k[0] + 1]++;
    }
    for (int a = 0; a < n; ++a) ctx->nc_start[a + 1] += ctx->nc_start[a];
    ctx->aotot.assign(n, 0);
    // Each atom's neighbours in descending order of their C block's upper
    // limit: surviving (F, G) terms then gather in the leading rows and
    // columns of the D_AB products, so whole tiles can be skipped.
    std::vector<double> cmax(C.keys.size());
    if (!C.keys.empty()) {
      CK(cudaMemcpyAsync(cmax.data(), C.maxabs.p, sizeof(double) * C.keys.size(),
                         cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
    }
    std::vector<int64_t> order(C.keys.size());
    for (size_t e = 0; e < order.size(); ++e) order[e] = (int64_t)e;
    for (int a = 0; a < n; ++a)
      std::stable_sort(order.begin() + ctx->nc_start[a], order.begin() + ctx->nc_start[a + 1],
                       [&](int64_t x, int64_t y) { return cmax[x] > cmax[y]; });
    for (size_t q = 0; q < C.keys.size(); ++q) {  // keys sorted: grouped by atom
      const int64_t e = order[q];
      int32_t k[5];
      hk_unpack(C.keys[e], k);
      NbrEntry &ne = ctx->nbr[q];
      ne.other = k[1];
      ne.n[0] = k[2]; ne.n[1] = k[3]; ne.n[2] = k[4];
      ne.aopre = (int32_t)ctx->aotot[k[0]];
      ne.pad = 0;
      ne.cblk = e;
      ctx->aotot[k[0]] += ctx->nao[k[1]];
    }
    ctx->items.resize(V.keys.size());
    int64_t wg = 0, wf = 0, mk = 0;
    for (size_t e = 0; e < V.keys.size(); ++e) {
      int32_t k[5];
      hk_unpack(V.keys[e], k);
      WorkItem &it = ctx->items[e];
      it.a = k[0]; it.b = k[1];
      it.n[0] = k[2]; it.n[1] = k[3]; it.n[2] = k[4];
      it.nF = (int32_t)(ctx->nc_start[k[0] + 1] - ctx->nc_start[k[0]]);
      it.nG = (int32_t)(ctx->nc_start[k[1] + 1] - ctx->nc_start[k[1]]);
      it.nFw = (it.nF + 31) / 32;
      it.vblk = (int64_t)e;
      it.dab = -1;
      it.fbase = ctx->nc_start[k[0]];
      it.gbase = ctx->nc_start[k[1]];
      it.mask_off = mk;
      it.wg_off = wg;
      it.wf_off = wf;
      // role of the pair under the mirror map <A,B> -> <B,A>
      const bool self = k[0] == k[1] && k[2] == 0 && k[3] == 0 && k[4] == 0;
      const bool canon = k[0] < k[1] || (k[0] == k[1] && std::make_tuple(k[2], k[3], k[4]) >
                                                             std::make_tuple(0, 0, 0));
      it.role = self ? 0 : canon ? 1 : 2;
      it.pad = 0;
      mk += (int64_t)it.nG * 4 * it.nFw;
      wg += it.nG;
      wf += it.nF;
    }
    ctx->nwg = wg;
    ctx->nwf = wf;
    ctx->nmask = mk;
    std::vector<int32_t> ncol(ctx->aotot.begin(), ctx->aotot.end());
    CK(ctx->d_ncol.reserve(n));
    CK(cudaMemcpyAsync(ctx->d_ncol.p, ncol.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    CK(ctx->d_nbr.reserve(ctx->nbr.size()));
    if (!ctx->nbr.empty())
      CK(cudaMemcpyAsync(ctx->d_nbr.p, ctx->nbr.data(), sizeof(NbrEntry) * ctx->nbr.size(),
                         cudaMemcpyHostToDevice, st));
  }
  if (cv_changed || D.keys_changed) {
    ctx->dindex.clear();
    ctx->dindex.reserve(D.keys.size() * 2);
    std::vector<int64_t> vals(D.keys.size());
    for (size_t e = 0; e < D.keys.size(); ++e) {
      ctx->dindex[D.keys[e]] = (int64_t)e;
      vals[e] = (int64_t)e;
    }
    std::vector<uint64_t> tk;
    std::vector<int64_t> tv;
    build_table(D.keys, vals, tk, tv, ctx->dmask);
    CK(ctx->d_dhkeys.reserve(tk.size()));
    CK(ctx->d_dhvals.reserve(tv.size()));
    CK(cudaMemcpyAsync(ctx->d_dhkeys.p, tk.data(), sizeof(uint64_t) * tk.size(),
                       cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ctx->d_dhvals.p, tv.data(), sizeof(int64_t) * tv.size(),
                       cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));  // tk, tv are about to go out of scope
    for (auto &it : ctx->items) {
      auto f = ctx->dindex.find(hk_pack(it.a, it.b, it.n[0], it.n[1], it.n[2]));
      it.dab = f == ctx->dindex.end() ? -1 : f->second;
    }
    CK(ctx->d_items.reserve(ctx->items.size()));
    if (!ctx->items.empty())
      CK(cudaMemcpyAsync(ctx->d_items.p, ctx->items.data(), sizeof(WorkItem) * ctx->items.size(),
                         cudaMemcpyHostToDevice, st));
  }
  C.keys_changed = V.keys_changed = D.keys_changed = false;
  ctx->plan_valid = true;
  return HFX_OK;
}

// Bitwise check that every block of kind k has its mirror key (j, i, -n) and
// that the mirror equals its transpose.
hfx_status check_mirror(hfx_ctx *ctx, int k, bool *ok) {
  Kind &K = ctx->K[k];
  cudaStream_t st = ctx->stream;
  const int64_t n = (int64_t)K.keys.size();
  std::vector<int64_t> mir(n);
  std::vector<int32_t> rows(n);
  for (int64_t e = 0; e < n; ++e) {
    int32_t q[5];
    hk_unpack(K.keys[e], q);
    const uint64_t mk = hk_pack(q[1], q[0], -q[2], -q[3], -q[4]);
    auto it = std::lower_bound(K.keys.begin(), K.keys.end(), mk);
    mir[e] = (it != K.keys.end() && *it == mk) ? (int64_t)(it - K.keys.begin()) : -1;
    rows[e] = k == 1 ? ctx->nabf[q[0]] : ctx->nao[q[0]];
  }
  int64_t *d_mir = nullptr;
  int32_t *d_rows = nullptr;
  unsigned *d_bad = nullptr;
  CK(cudaMalloc((void **)&d_mir, sizeof(int64_t) * (n ? n : 1)));
  CK(cudaMalloc((void **)&d_rows, sizeof(int32_t) * (n ? n : 1)));
  CK(cudaMalloc((void **)&d_bad, sizeof(unsigned)));
  CK(cudaMemsetAsync(d_bad, 0, sizeof(unsigned), st));
  CK(cudaMemcpyAsync(d_mir, mir.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d_rows, rows.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
  CK(launch_check_mirror(K.data.p, K.d_offs.p, d_mir, d_rows, n, d_bad, st));
  ctx->launches += n > 0;
  unsigned bad = 0;
  CK(cudaMemcpyAsync(&bad, d_bad, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  cudaFree(d_mir);
  cudaFree(d_rows);
  cudaFree(d_bad);
  *ok = bad == 0;
  return HFX_OK;
}

// Digit-sliced C (two layouts) and V for the split-precision products.
hfx_status split_prepare(hfx_ctx *ctx, int ks) {
  cudaStream_t st = ctx->stream;
  const int n = ctx->natoms;
  const int64_t nv = (int64_t)ctx->items.size();
  const int TM = 128, NT = 64, TK = 32;
  ctx->ktY.assign(n, 0);
  ctx->kt4.assign(n, 0);
  std::vector<int64_t> cy_base(n + 1, 0), cy_row(n + 1, 0), c4_base(n + 1, 0), c4_row(n + 1, 0);
  for (int x = 0; x < n; ++x) {
    const int64_t nx = ctx->nao[x], px = ctx->nabf[x], ncol = ctx->aotot[x];
    ctx->ktY[x] = (int32_t)((px + TK - 1) / TK);
    ctx->kt4[x] = (int32_t)((px * nx + TK - 1) / TK);
    const int64_t mty = (nx * ncol + TM - 1) / TM, mt4 = (ncol + TM - 1) / TM;
    cy_row[x + 1] = cy_row[x] + mty * TM;
    c4_row[x + 1] = c4_row[x] + mt4 * TM;
    cy_base[x + 1] = cy_base[x] + mty * ctx->ktY[x] * ks * TM * TK;
    c4_base[x + 1] = c4_base[x] + mt4 * ctx->kt4[x] * ks * TM * TK;
  }
  std::vector<int64_t> vs_base(nv + 1, 0), v_row(nv + 1, 0);
  for (int64_t e = 0; e < nv; ++e) {
    const WorkItem &it = ctx->items[e];
    const int64_t ntv = (ctx->nabf[it.a] + NT - 1) / NT;
    v_row[e + 1] = v_row[e] + ntv * NT;
    vs_base[e + 1] = vs_base[e] + ntv * ctx->ktY[it.b] * ks * NT * TK;
  }
  // C as rows (al, a), K = F blocks of width 16 or 32
  std::vector<int64_t> cz_base(n + 1, 0), cz_row(n + 1, 0);
  std::vector<int32_t> kofs(ctx->nbr.size()), ktotZ(n);
  for (int x = 0; x < n; ++x) {
    int32_t k = 0;
    for (int64_t q = ctx->nc_start[x]; q < ctx->nc_start[x + 1]; ++q) {
      kofs[q] = k;
      k += ctx->nao[ctx->nbr[q].other] <= 16 ? 16 : 32;
    }
    ktotZ[x] = k;
    const int64_t mtz = ((int64_t)ctx->nabf[x] * ctx->nao[x] + TM - 1) / TM;
    cz_row[x + 1] = cz_row[x] + mtz * TM;
    cz_base[x + 1] = cz_base[x] + mtz * (int64_t)k * ks * TM;
  }
  ctx->h_cz_rows = cz_row[n];
  CK(ctx->d_cz.reserve(cz_base[n]));
  CK(ctx->d_cz_e.reserve(cz_row[n]));
  std::vector<int64_t> czm(cz_base);
  czm.insert(czm.end(), cz_row.begin(), cz_row.end());
  CK(ctx->d_cz_meta.reserve(czm.size()));
  CK(cudaMemcpyAsync(ctx->d_cz_meta.p, czm.data(), sizeof(int64_t) * czm.size(),
                     cudaMemcpyHostToDevice, st));
  CK(ctx->d_kofs.reserve(std::max<size_t>(kofs.size(), 1)));
  CK(ctx->d_ktotZ.reserve(n));
  if (!kofs.empty())
    CK(cudaMemcpyAsync(ctx->d_kofs.p, kofs.data(), sizeof(int32_t) * kofs.size(),
                       cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ctx->d_ktotZ.p, ktotZ.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
  ctx->ktotZ_h = ktotZ;
  CK(cudaStreamSynchronize(st));
  // column (G, g) of an atom's concatenated neighbour blocks -> local index of G
  {
    std::vector<int64_t> coloff(n + 1, 0);
    for (int x = 0; x < n; ++x) coloff[x + 1] = coloff[x] + ctx->aotot[x];
    std::vector<int16_t> colG(std::max<int64_t>(coloff[n], 1));
    for (int x = 0; x < n; ++x)
      for (int64_t q = ctx->nc_start[x]; q < ctx->nc_start[x + 1]; ++q) {
        const NbrEntry &e = ctx->nbr[q];
        for (int g = 0; g < ctx->nao[e.other]; ++g)
          colG[coloff[x] + e.aopre + g] = (int16_t)(q - ctx->nc_start[x]);
      }
    CK(ctx->d_colG.reserve(colG.size()));
    CK(ctx->d_coloff.reserve(n + 1));
    CK(cudaMemcpyAsync(ctx->d_colG.p, colG.data(), sizeof(int16_t) * colG.size(),
                       cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ctx->d_coloff.p, coloff.data(), sizeof(int64_t) * (n + 1),
                       cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
  }
  ctx->h_cy_rows = cy_row[n];
  ctx->h_c4_rows = c4_row[n];
  ctx->h_v_rows = v_row[nv];
  CK(ctx->d_cy.reserve(cy_base[n]));
  CK(ctx->d_c4.reserve(c4_base[n]));
  CK(ctx->d_vs.reserve(vs_base[nv]));
  CK(ctx->d_cy_e.reserve(cy_row[n]));
  CK(ctx->d_c4_e.reserve(c4_row[n]));
  CK(ctx->d_vs_e.reserve(v_row[nv]));
  std::vector<int64_t> meta;
  meta.insert(meta.end(), cy_base.begin(), cy_base.end());
  meta.insert(meta.end(), cy_row.begin(), cy_row.end());
  meta.insert(meta.end(), c4_base.begin(), c4_base.end());
  meta.insert(meta.end(), c4_row.begin(), c4_row.end());
  meta.insert(meta.end(), vs_base.begin(), vs_base.end());
  meta.insert(meta.end(), v_row.begin(), v_row.end());
  meta.insert(meta.end(), ctx->nc_start.begin(), ctx->nc_start.end());
  CK(ctx->d_split_meta.reserve(meta.size()));
  CK(cudaMemcpyAsync(ctx->d_split_meta.p, meta.data(), sizeof(int64_t) * meta.size(),
                     cudaMemcpyHostToDevice, st));
  std::vector<int32_t> kt(ctx->ktY);
  kt.insert(kt.end(), ctx->kt4.begin(), ctx->kt4.end());
  CK(ctx->d_kt.reserve(kt.size()));
  CK(cudaMemcpyAsync(ctx->d_kt.p, kt.data(), sizeof(int32_t) * kt.size(), cudaMemcpyHostToDevice,
                     st));
  CK(cudaStreamSynchronize(st));
  ctx->split_ks = ks;
  return HFX_OK;
}

// D digit-tile layout: per D block (i, j, n) a [ks][R x kb] tile, R = 16 or
// 32 rows (nao(j)), kb = 16 or 32 (nao(i)); per (atom, ao) column maxima.
hfx_status dz_prepare_meta(hfx_ctx *ctx, int ks) {
  cudaStream_t st = ctx->stream;
  const Kind &D = ctx->K[2];
  const int64_t nd = (int64_t)D.keys.size();
  const int n = ctx->natoms;
  std::vector<int64_t> off(nd + 1, 0);
  std::vector<int32_t> ij(2 * nd);
  for (int64_t e = 0; e < nd; ++e) {
    int32_t q[5];
    hk_unpack(D.keys[e], q);
    ij[2 * e] = q[0];
    ij[2 * e + 1] = q[1];
    const int64_t R = ctx->nao[q[1]] <= 16 ? 16 : 32, kb = ctx->nao[q[0]] <= 16 ? 16 : 32;
    off[e + 1] = off[e] + (int64_t)ks * R * kb;
  }
  std::vector<int32_t> aoff(n + 1, 0);
  int kbmax = 16, naomax = 1, naomin = 1 << 30;
  for (int x = 0; x < n; ++x) {
    aoff[x + 1] = aoff[x] + ctx->nao[x];
    if (ctx->nao[x] > 16) kbmax = 32;
    if (ctx->nao[x] > 32)
      return fail(ctx, HFX_E_ARG, "the split modes support at most 32 NAOs per atom");
    naomax = std::max(naomax, ctx->nao[x]);
    naomin = std::min(naomin, ctx->nao[x]);
  }
  // staged Y rows per tile: al rows spanned by 128 (al, a) rows, all b (plus
  // 2 pairs of padding per al), the 16-column blocks of one G; for the small
  // class (jobs whose blocks have at most 16 AOs) with the largest such atom
  int naosmall = 1;
  for (int x = 0; x < n; ++x)
    if (ctx->nao[x] <= 16) naosmall = std::max(naosmall, ctx->nao[x]);
  ctx->zc_shape = ZcPlanShape{kbmax, naomax,
                              (127 / naomin + 2) * (naomax * 16 + 2) * 8 * ((naomax + 15) / 16),
                              (127 / naomin + 2) * (naosmall * 16 + 2) * 8};
  CK(ctx->d_dz.reserve(std::max<int64_t>(off[nd], 1)));
  CK(ctx->d_dz_off.reserve(std::max<int64_t>(nd, 1)));
  CK(ctx->d_dij.reserve(std::max<int64_t>(2 * nd, 1)));
  CK(ctx->d_aoff.reserve(n + 1));
  CK(ctx->d_de.reserve(std::max<int32_t>(aoff[n], 1)));
  // zero tile: up to 6 digits of a 32 x 32 tile
  CK(ctx->d_dzero.reserve(6 * 32 * 32));
  CK(cudaMemsetAsync(ctx->d_dzero.p, 0, 6 * 32 * 32 * sizeof(__nv_bfloat16), st));
  if (nd) {
    CK(cudaMemcpyAsync(ctx->d_dz_off.p, off.data(), sizeof(int64_t) * nd, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ctx->d_dij.p, ij.data(), sizeof(int32_t) * 2 * nd, cudaMemcpyHostToDevice, st));
  }
  CK(cudaMemcpyAsync(ctx->d_aoff.p, aoff.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  ctx->dz_nd = nd;
  ctx->dz_ks = ks;
  ctx->kbmax = kbmax;
  if (!ctx->nsm) {
    int dev = 0, sm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev));
    ctx->nsm = sm;
  }
  return HFX_OK;
}

SplitShared split_shared(hfx_ctx *ctx) {
  SplitShared S{};
  const int n = ctx->natoms;
  const int64_t nv = (int64_t)ctx->items.size();
  const int64_t *m = ctx->d_split_meta.p;
  S.natoms = n;
  S.nv = nv;
  S.nao = ctx->d_nao.p;
  S.nabf = ctx->d_nabf.p;
  S.ncol = ctx->d_ncol.p;
  S.ktY = ctx->d_kt.p;
  S.kt4 = ctx->d_kt.p + n;
  S.cy_base = m;
  S.cy_rowpre = m + (n + 1);
  S.c4_base = m + 2 * (n + 1);
  S.c4_rowpre = m + 3 * (n + 1);
  S.vs_base = m + 4 * (n + 1);
  S.v_rowpre = m + 4 * (n + 1) + (nv + 1);
  S.nc_start = m + 4 * (n + 1) + 2 * (nv + 1);
  S.nbr = ctx->d_nbr.p;
  S.items = ctx->d_items.p;
  S.Cd = ctx->K[0].data.p;
  S.Co = ctx->K[0].d_offs.p;
  S.Vd = ctx->K[1].data.p;
  S.Vo = ctx->K[1].d_offs.p;
  S.masks = ctx->d_masks.p;
  S.wg = ctx->d_wg.p;
  S.shash = DevHash{ctx->d_shkeys.p, ctx->d_shvals.p, ctx->smask};
  S.acc = ctx->d_acc.p;
  S.err = ctx->d_err.p;
  S.sym = ctx->sym ? 1 : 0;
  S.cy = ctx->d_cy.p;
  S.cy_e = ctx->d_cy_e.p;
  S.c4 = ctx->d_c4.p;
  S.c4_e = ctx->d_c4_e.p;
  S.vs = ctx->d_vs.p;
  S.vs_e = ctx->d_vs_e.p;
  S.h_cy_rows = ctx->h_cy_rows;
  S.h_c4_rows = ctx->h_c4_rows;
  S.h_v_rows = ctx->h_v_rows;
  S.cz = ctx->d_cz.p;
  S.cz_e = ctx->d_cz_e.p;
  S.cz_base = ctx->d_cz_meta.p;
  S.cz_rowpre = ctx->d_cz_meta.p + (n + 1);
  S.kofs = ctx->d_kofs.p;
  S.ktotZ = ctx->d_ktotZ.p;
  S.Dd = ctx->K[2].data.p;
  S.Do = ctx->K[2].d_offs.p;
  S.dhash = DevHash{ctx->d_dhkeys.p, ctx->d_dhvals.p, ctx->dmask};
  S.h_cz_rows = ctx->h_cz_rows;
  S.dz = ctx->d_dz.p;
  S.dzero = ctx->d_dzero.p;
  S.dz_off = ctx->d_dz_off.p;
  S.dij = ctx->d_dij.p;
  S.de = ctx->d_de.p;
  S.aoff = ctx->d_aoff.p;
  S.h_nd = ctx->dz_nd > 0 ? ctx->dz_nd : 0;
  S.colG = ctx->d_colG.p;
  S.coloff = ctx->d_coloff.p;
  S.nsm = ctx->nsm;
  {
    // P of the D_AB piece: at least one g column of P (K = nabf nao of A) and
    // of the staged Y (nabf(A) nao(B) rows) at a time
    int64_t kmax = 0, pmax = 0, nmax = 0;
    for (int x = 0; x < ctx->natoms; ++x) {
      kmax = std::max<int64_t>(kmax, (int64_t)ctx->nabf[x] * ctx->nao[x]);
      pmax = std::max<int64_t>(pmax, ctx->nabf[x]);
      nmax = std::max<int64_t>(nmax, ctx->nao[x]);
    }
    S.pd_pairs = (int32_t)std::max<int64_t>(6400, kmax + pmax * nmax);
  }
  return S;
}

// Cauchy-Schwarz ERI bounds sqrt(max(Q, 0)) per C block (k_diag_eri): the
// V blocks XX, XY, YX, YY and the partner C block of every C block (x, y, n).
hfx_status eri_prepare(hfx_ctx *ctx) {
  const Kind &C = ctx->K[0], &V = ctx->K[1];
  cudaStream_t st = ctx->stream;
  const int64_t nC = (int64_t)C.keys.size();
  auto findk = [](const std::vector<uint64_t> &keys, uint64_t k) -> int64_t {
    auto it = std::lower_bound(keys.begin(), keys.end(), k);
    return (it != keys.end() && *it == k) ? (int64_t)(it - keys.begin()) : -1;
  };
  std::vector<int64_t> meta(5 * std::max<int64_t>(nC, 1), -1);
  std::vector<int32_t> cxy(2 * std::max<int64_t>(nC, 1), 0);
  for (int64_t e = 0; e < nC; ++e) {
    int32_t q[5];
    hk_unpack(C.keys[e], q);
    const int x = q[0], y = q[1];
    cxy[2 * e] = x;
    cxy[2 * e + 1] = y;
    meta[5 * e] = findk(V.keys, hk_pack(x, x, 0, 0, 0));
    const bool same = x == y && q[2] == 0 && q[3] == 0 && q[4] == 0;
    if (!same) {
      meta[5 * e + 1] = findk(V.keys, hk_pack(x, y, q[2], q[3], q[4]));
      meta[5 * e + 2] = findk(V.keys, hk_pack(y, x, -q[2], -q[3], -q[4]));
      meta[5 * e + 3] = findk(V.keys, hk_pack(y, y, 0, 0, 0));
      meta[5 * e + 4] = findk(C.keys, hk_pack(y, x, -q[2], -q[3], -q[4]));
    }
  }
  DevBuf<int64_t> d_meta;
  DevBuf<int32_t> d_cxy;
  CK(d_meta.reserve(meta.size()));
  CK(d_cxy.reserve(cxy.size()));
  CK(ctx->d_eri_sq.reserve(std::max<int64_t>(nC, 1)));
  CK(cudaMemcpyAsync(d_meta.p, meta.data(), sizeof(int64_t) * meta.size(), cudaMemcpyHostToDevice,
                     st));
  CK(cudaMemcpyAsync(d_cxy.p, cxy.data(), sizeof(int32_t) * cxy.size(), cudaMemcpyHostToDevice,
                     st));
  CK(launch_diag_eri(C.data.p, C.d_offs.p, V.data.p, V.d_offs.p, d_meta.p, d_cxy.p,
                     ctx->d_nao.p, ctx->d_nabf.p, nC, ctx->d_eri_sq.p, st));
  ctx->launches += nC > 0;
  CK(cudaStreamSynchronize(st));  // meta and cxy are freed on return
  ctx->eri_valid = true;
  return HFX_OK;
}

size_t scratch_budget_doubles() {
  size_t freeb = 0, totalb = 0;
  cudaMemGetInfo(&freeb, &totalb);
  size_t budget = std::min<size_t>((size_t)32 << 30, freeb * 2 / 5);
  if (const char *e = std::getenv("HFX_SCRATCH_MB")) {
    const long long mb = std::atoll(e);
    if (mb > 0) budget = (size_t)mb << 20;
  }
  return std::max<size_t>(budget / sizeof(double), 1);
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

hfx_status hfx_create(const double lattice[9], int32_t natoms, const double *pos,
                      const int32_t *species, int32_t nspecies, const int32_t *nao,
                      const int32_t *nabf, void *cuda_stream, hfx_ctx **out) {
  if (!out) return HFX_E_ARG;
  *out = nullptr;
  if (natoms <= 0 || natoms >= (1 << 20) || !species || nspecies <= 0 || !nao || !nabf)
    return HFX_E_ARG;
  for (int s = 0; s < nspecies; ++s)
    if (nao[s] < 1 || nao[s] > HFX_MAX_NAO || nabf[s] < 1 || nabf[s] > HFX_MAX_NABF)
      return HFX_E_ARG;
  for (int a = 0; a < natoms; ++a)
    if (species[a] < 0 || species[a] >= nspecies) return HFX_E_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return HFX_E_CUDA;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess || prop.major < 10) return HFX_E_CUDA;
  hfx_ctx *ctx = new (std::nothrow) hfx_ctx();
  if (!ctx) return HFX_E_NOMEM;
  ctx->natoms = natoms;
  ctx->nao.resize(natoms);
  ctx->nabf.resize(natoms);
  for (int a = 0; a < natoms; ++a) {
    ctx->nao[a] = nao[species[a]];
    ctx->nabf[a] = nabf[species[a]];
  }
  if (lattice) std::memcpy(ctx->lattice, lattice, sizeof(ctx->lattice));
  if (pos) ctx->pos.assign(pos, pos + 3 * (size_t)natoms);
  ctx->stream = (cudaStream_t)cuda_stream;
  ctx->K[0].name = 'C';
  ctx->K[1].name = 'V';
  ctx->K[2].name = 'D';
  hfx_status s = HFX_OK;
  if (ctx->d_nao.reserve(natoms) != cudaSuccess || ctx->d_nabf.reserve(natoms) != cudaSuccess ||
      ctx->d_err.reserve(1) != cudaSuccess || ctx->d_counters.reserve(8) != cudaSuccess ||
      ctx->d_ex.reserve(1) != cudaSuccess || ctx->d_collect.reserve(1) != cudaSuccess ||
      ctx->d_counters.reserve(24) != cudaSuccess)
    s = HFX_E_NOMEM;
  if (s == HFX_OK &&
      (cudaMemcpy(ctx->d_nao.p, ctx->nao.data(), sizeof(int32_t) * natoms,
                  cudaMemcpyHostToDevice) != cudaSuccess ||
       cudaMemcpy(ctx->d_nabf.p, ctx->nabf.data(), sizeof(int32_t) * natoms,
                  cudaMemcpyHostToDevice) != cudaSuccess ||
       cudaMemset(ctx->d_err.p, 0, sizeof(unsigned)) != cudaSuccess))
    s = HFX_E_CUDA;
  for (int e = 0; s == HFX_OK && e < 5; ++e)
    if (cudaEventCreate(&ctx->ev[e]) != cudaSuccess) s = HFX_E_CUDA;
  for (int e = 0; s == HFX_OK && e < 10; ++e)
    if (cudaEventCreate(&ctx->kev[e]) != cudaSuccess) s = HFX_E_CUDA;
  for (int e = 0; s == HFX_OK && e < 4; ++e)
    if (cudaEventCreate(&ctx->sev[e]) != cudaSuccess) s = HFX_E_CUDA;
  if (s != HFX_OK) {
    hfx_destroy(ctx);
    return s;
  }
  *out = ctx;
  return HFX_OK;
}

void hfx_destroy(hfx_ctx *ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (auto &e : ctx->ev)
    if (e) cudaEventDestroy(e);
  for (auto &e : ctx->kev)
    if (e) cudaEventDestroy(e);
  for (auto &e : ctx->sev)
    if (e) cudaEventDestroy(e);
  delete ctx;
}

const char *hfx_last_error(const hfx_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

static hfx_status set_one(hfx_ctx *ctx, int k, int32_t i, int32_t j, const int32_t n[3],
                          const double *blk) {
  if (!ctx) return HFX_E_ARG;
  if (!n || !blk) return fail(ctx, HFX_E_ARG, "null pointer");
  const int32_t key[5] = {i, j, n[0], n[1], n[2]};
  if (!key_ok(ctx, key)) return fail(ctx, HFX_E_ARG, "block key out of range");
  Kind &K = ctx->K[k];
  const int64_t len = block_len(ctx, k, i, j);
  for (int64_t t = 0; t < len; ++t)
    if (!std::isfinite(blk[t])) return fail(ctx, HFX_E_ARG, "non-finite value in block");
  const uint64_t hk = hk_pack(i, j, n[0], n[1], n[2]);
  const bool is_new = K.map.find(hk) == K.map.end();
  Entry en{-1, (int64_t)K.pending.size(), len};
  K.pending.insert(K.pending.end(), blk, blk + len);
  K.map[hk] = en;
  invalidate(ctx, k, is_new);
  return HFX_OK;
}

hfx_status hfx_set_C(hfx_ctx *ctx, int32_t a, int32_t f, const int32_t n[3], const double *blk) {
  return set_one(ctx, 0, a, f, n, blk);
}
hfx_status hfx_set_V(hfx_ctx *ctx, int32_t a, int32_t b, const int32_t n[3], const double *blk) {
  return set_one(ctx, 1, a, b, n, blk);
}
hfx_status hfx_set_D(hfx_ctx *ctx, int32_t k, int32_t l, const int32_t n[3], const double *blk) {
  return set_one(ctx, 2, k, l, n, blk);
}

hfx_status hfx_set_many(hfx_ctx *ctx, char which, int64_t nblk, const int32_t *keys,
                        const double *data, const int64_t *offs, int on_device) {
  if (!ctx) return HFX_E_ARG;
  const int k = kind_index(which);
  if (k < 0) return fail(ctx, HFX_E_ARG, "which must be 'C', 'V' or 'D'");
  if (nblk < 0 || (nblk > 0 && (!keys || !data || !offs)))
    return fail(ctx, HFX_E_ARG, "null pointer or negative count");
  if (nblk == 0) return HFX_OK;
  if (offs[0] < 0) return fail(ctx, HFX_E_SHAPE, "negative offset");
  for (int64_t e = 0; e < nblk; ++e) {
    const int32_t *kk = keys + 5 * e;
    if (!key_ok(ctx, kk)) return fail(ctx, HFX_E_ARG, "block key out of range");
    if (offs[e + 1] - offs[e] != block_len(ctx, k, kk[0], kk[1]))
      return fail(ctx, HFX_E_SHAPE, "block size does not match nao/nabf");
  }
  Kind &K = ctx->K[k];
  const int64_t lo = offs[0], hi = offs[nblk];
  // A full re-set of a packed kind in its packed key order with the same
  // block sizes (C, V or D of the next SCF step): the values are copied into
  // the packed array in place, with no new chunk to allocate and no old one
  // to free, and the key map stays as it is.
  if (!K.dirty && K.data_is_chunk && K.chunks.size() == 1 && K.data.p == K.chunks[0].dev &&
      (int64_t)K.keys.size() == nblk && K.chunks[0].n == (size_t)(hi - lo)) {
    bool same = true;
    for (int64_t b = 0; same && b < nblk; ++b) {
      const int32_t *kk = keys + 5 * b;
      same = hk_pack(kk[0], kk[1], kk[2], kk[3], kk[4]) == K.keys[b] &&
             offs[b] - lo == K.offs[b];
    }
    if (same) {
      invalidate(ctx, k, false);
      cudaError_t e = cudaMemcpyAsync(K.chunks[0].dev, data + lo, (size_t)(hi - lo) * sizeof(double),
                                      on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                      ctx->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
      if (e != cudaSuccess) return fail_cuda(ctx, "cudaMemcpyAsync", e);
      return HFX_OK;
    }
  }
  Chunk c;
  c.n = (size_t)(hi - lo);
  cudaError_t e = cudaMalloc((void **)&c.dev, (c.n > 0 ? c.n : 1) * sizeof(double));
  if (e != cudaSuccess) return fail_cuda(ctx, "cudaMalloc", e);
  e = cudaMemcpyAsync(c.dev, data + lo, c.n * sizeof(double),
                      on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    cudaFree(c.dev);
    return fail_cuda(ctx, "cudaMemcpyAsync", e);
  }
  const int32_t id = (int32_t)K.chunks.size();
  K.chunks.push_back(c);
  bool any_new = false;
  for (int64_t b = 0; b < nblk; ++b) {
    const int32_t *kk = keys + 5 * b;
    const uint64_t hk = hk_pack(kk[0], kk[1], kk[2], kk[3], kk[4]);
    auto it = K.map.find(hk);
    if (it == K.map.end()) any_new = true;
    K.map[hk] = Entry{id, offs[b] - lo, offs[b + 1] - offs[b]};
  }
  invalidate(ctx, k, any_new);
  return HFX_OK;
}

hfx_status hfx_clear(hfx_ctx *ctx, char which) {
  if (!ctx) return HFX_E_ARG;
  const int k = kind_index(which);
  if (k < 0) return fail(ctx, HFX_E_ARG, "which must be 'C', 'V' or 'D'");
  Kind &K = ctx->K[k];
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  K.map.clear();
  K.pending.clear();
  if (K.data_is_chunk) {
    K.data.p = nullptr;
    K.data.n = 0;
    K.data_is_chunk = false;
  }
  K.free_chunks();
  invalidate(ctx, k, true);
  return HFX_OK;
}

hfx_status hfx_build(hfx_ctx *ctx, double theta, hfx_prec prec, int32_t nslices, double *ex_out) {
  if (!ctx) return HFX_E_ARG;
  if (!(theta >= 0.0) || !std::isfinite(theta)) return fail(ctx, HFX_E_ARG, "theta must be >= 0");
  // HFX_BF16X3 is the split path with two digits per operand: of the digit
  // products only hi*hi, hi*lo and lo*hi (orders 0 and 1) are formed
  const bool split = prec == HFX_OZAKI || prec == HFX_BF16X3;
  if (prec != HFX_FP64 && !split)
    return fail(ctx, HFX_E_ARG, "unknown precision mode");
  if (prec == HFX_BF16X3) {
    if (nslices != 0 && nslices != 2)
      return fail(ctx, HFX_E_ARG, "HFX_BF16X3 uses two digit slices (pass 0 or 2)");
    nslices = 2;
  }
  if (prec == HFX_OZAKI && nslices == 0) nslices = 6;
  if (prec == HFX_OZAKI && (nslices < 4 || nslices > 6))
    return fail(ctx, HFX_E_ARG, "HFX_OZAKI takes 4 to 6 digit slices");
  for (int k = 0; k < 3; ++k)
    if (ctx->K[k].map.empty())
      return fail(ctx, HFX_E_STATE, std::string("no ") + ctx->K[k].name + " blocks set");
  ctx->results_valid = false;
  ctx->from_batch = false;
  ctx->launches = 0;
  double kms[8] = {0};
  cudaStream_t st = ctx->stream;
  if (!ctx->theta_atom.empty()) {
    CK(ctx->d_theta_atom.reserve(ctx->theta_atom.size()));
    CK(cudaMemcpyAsync(ctx->d_theta_atom.p, ctx->theta_atom.data(),
                       sizeof(double) * ctx->theta_atom.size(), cudaMemcpyHostToDevice, st));
  }
  CK(cudaEventRecord(ctx->ev[0], st));
  CK(cudaMemsetAsync(ctx->d_err.p, 0, sizeof(unsigned), st));
  const bool vd_dirty = ctx->K[1].dirty || ctx->K[2].dirty;
  const bool cv_dirty = ctx->K[0].dirty || ctx->K[1].dirty || !ctx->plan_valid;
  ctx->c_reordered = ctx->K[0].dirty;
  for (int k = 0; k < 3; ++k) {
    hfx_status s = pack_kind(ctx, k);
    if (s != HFX_OK) return s;
  }
  if (vd_dirty) {
    bool okV = false, okD = false;
    hfx_status s = check_mirror(ctx, 1, &okV);
    if (s == HFX_OK) s = check_mirror(ctx, 2, &okD);
    if (s != HFX_OK) return s;
    const char *no = std::getenv("HFX_NO_MIRROR");
    ctx->sym = okV && okD && !(no && no[0] && no[0] != '0');
  }
  {
    unsigned perr = 0;
    CK(cudaMemcpyAsync(&perr, ctx->d_err.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (perr & HFX_DEV_ERR_NONFINITE) {
      for (int k = 0; k < 3; ++k) ctx->K[k].dirty = true;  // re-check on the next build
      return fail(ctx, HFX_E_ARG, "non-finite value in an input block");
    }
    hfx_status s = build_plan(ctx);
    if (s != HFX_OK) return s;
  }
  if (ctx->eps_eri >= 0.0 && !ctx->eri_valid) {
    hfx_status s = eri_prepare(ctx);
    if (s != HFX_OK) return s;
  }
  // ---- screen (retry with a larger Sigma key table on overflow)
  CK(ctx->d_masks.reserve(ctx->nmask));
  CK(ctx->d_wg.reserve(ctx->nwg));
  CK(ctx->d_wf.reserve(ctx->nwf));
  if (ctx->stab_cap == 0)
    ctx->stab_cap = pow2_at_least(64 * (uint64_t)ctx->K[0].keys.size() + 1024);
  unsigned long long counters[24] = {0};
  unsigned herr = 0;
  for (int attempt = 0;; ++attempt) {
    CK(ctx->d_stab.reserve(ctx->stab_cap));
    CK(cudaMemsetAsync(ctx->d_stab.p, 0xFF, sizeof(unsigned long long) * ctx->stab_cap, st));
    CK(cudaMemsetAsync(ctx->d_wg.p, 0, ctx->nwg ? ctx->nwg : 1, st));
    CK(cudaMemsetAsync(ctx->d_wf.p, 0, sizeof(uint32_t) * (ctx->nwf ? ctx->nwf : 1), st));
    CK(cudaMemsetAsync(ctx->d_counters.p, 0, sizeof(unsigned long long) * 24, st));
    CK(cudaMemsetAsync(ctx->d_err.p, 0, sizeof(unsigned), st));
    ScreenArgs a{};
    a.items = ctx->d_items.p;
    a.nitems = (int64_t)ctx->items.size();
    a.nwg = ctx->nwg;
    a.nbr = ctx->d_nbr.p;
    a.nao = ctx->d_nao.p;
    a.nabf = ctx->d_nabf.p;
    a.C = DevBlocks{ctx->K[0].data.p, ctx->K[0].d_offs.p, ctx->K[0].maxabs.p};
    a.V = DevBlocks{ctx->K[1].data.p, ctx->K[1].d_offs.p, ctx->K[1].maxabs.p};
    a.D = DevBlocks{ctx->K[2].data.p, ctx->K[2].d_offs.p, ctx->K[2].maxabs.p};
    a.dhash = DevHash{ctx->d_dhkeys.p, ctx->d_dhvals.p, ctx->dmask};
    a.theta = theta;
    a.masks = ctx->d_masks.p;
    a.wg_flags = ctx->d_wg.p;
    a.wf_flags = ctx->d_wf.p;
    a.sig_keys = ctx->d_stab.p;
    a.sig_mask = ctx->stab_cap - 1;
    a.sig_count = ctx->d_counters.p + 7;
    a.sig_limit = ctx->stab_cap / 2;
    a.counters = ctx->d_counters.p;
    a.eri_sq = ctx->eps_eri >= 0.0 ? ctx->d_eri_sq.p : nullptr;
    a.theta_atom = ctx->theta_atom.empty() ? nullptr : ctx->d_theta_atom.p;
    a.eps_eri = ctx->eps_eri;
    a.err = ctx->d_err.p;
    CK(cudaEventRecord(ctx->kev[8], st));
    CK(launch_screen(a, st));
    CK(cudaEventRecord(ctx->kev[9], st));
    ctx->launches += a.nwg > 0;
    CK(cudaMemcpyAsync(counters, ctx->d_counters.p, sizeof(counters), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&herr, ctx->d_err.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if ((herr & HFX_DEV_ERR_HASH_FULL) && attempt < 6) {
      ctx->stab_cap *= 4;
      continue;
    }
    if (herr) return fail(ctx, HFX_E_CUDA, "screen kernel reported error " + std::to_string(herr));
    float ms = 0;
    cudaEventElapsedTime(&ms, ctx->kev[8], ctx->kev[9]);
    kms[0] = ms;
    break;
  }
  // ---- Sigma key set: collect, sort, offsets, lookup table
  const int64_t nsig = (int64_t)counters[7];
  {
    CK(ctx->d_collect.reserve(nsig + 1));
    CK(cudaMemsetAsync(ctx->d_counters.p + 7, 0, sizeof(unsigned long long), st));
    CK(launch_collect_keys(ctx->d_stab.p, ctx->stab_cap, ctx->d_collect.p,
                           ctx->d_counters.p + 7, st));
    ctx->launches += 1;
    ctx->sig_keys.resize(nsig);
    if (nsig)
      CK(cudaMemcpyAsync(ctx->sig_keys.data(), ctx->d_collect.p, sizeof(uint64_t) * nsig,
                         cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    std::sort(ctx->sig_keys.begin(), ctx->sig_keys.end());
    ctx->sig_offs.assign(nsig + 1, 0);
    for (int64_t e = 0; e < nsig; ++e) {
      int32_t k[5];
      hk_unpack(ctx->sig_keys[e], k);
      ctx->sig_offs[e + 1] = ctx->sig_offs[e] + (int64_t)ctx->nao[k[0]] * ctx->nao[k[1]];
    }
    std::vector<uint64_t> tk;
    std::vector<int64_t> tv;
    std::vector<int64_t> vals(ctx->sig_offs.begin(), ctx->sig_offs.end() - 1);
    build_table(ctx->sig_keys, vals, tk, tv, ctx->smask);
    CK(ctx->d_shkeys.reserve(tk.size()));
    CK(ctx->d_shvals.reserve(tv.size()));
    CK(ctx->d_skeys.reserve(nsig));
    CK(ctx->d_soffs.reserve(nsig + 1));
    CK(cudaMemcpyAsync(ctx->d_shkeys.p, tk.data(), sizeof(uint64_t) * tk.size(),
                       cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ctx->d_shvals.p, tv.data(), sizeof(int64_t) * tv.size(),
                       cudaMemcpyHostToDevice, st));
    if (nsig)
      CK(cudaMemcpyAsync(ctx->d_skeys.p, ctx->sig_keys.data(), sizeof(uint64_t) * nsig,
                         cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ctx->d_soffs.p, ctx->sig_offs.data(), sizeof(int64_t) * (nsig + 1),
                       cudaMemcpyHostToDevice, st));
    const int64_t nelem = ctx->sig_offs[nsig];
    CK(ctx->d_acc.reserve(2 * nelem));
    CK(cudaMemsetAsync(ctx->d_acc.p, 0, sizeof(unsigned long long) * 2 * (nelem ? nelem : 1), st));
    CK(cudaStreamSynchronize(st));  // tk, tv, vals go out of scope
  }
  SplitShared SS{};
  if (split) {
    if (cv_dirty || ctx->split_ks != nslices) {
      hfx_status s = split_prepare(ctx, nslices);
      if (s != HFX_OK) return s;
      SS = split_shared(ctx);
      CK(split_slice_inputs(SS, nslices, st));
      CK(split_slice_cz(SS, nslices, st));
      ctx->launches += (SS.h_cy_rows > 0) + (SS.h_c4_rows > 0) + (SS.h_v_rows > 0) +
                       (SS.h_cz_rows > 0);
    }
    if (ctx->dz_nd < 0 || ctx->dz_ks != nslices) {
      hfx_status s = dz_prepare_meta(ctx, nslices);
      if (s != HFX_OK) return s;
    }
    SS = split_shared(ctx);
    // D digit tiles (D may change every build)
    CK(cudaMemsetAsync(ctx->d_de.p, 0, sizeof(unsigned long long) *
                                           std::max<size_t>(ctx->d_de.n, 1), st));
    CK(split_dz_prepare(SS, nslices, st));
    ctx->launches += 2 * (SS.h_nd > 0);
    CK(ctx->d_njobs.reserve(4));
    CK(ctx->d_tmacs.reserve(4));
  }
  double tmac_y = 0, tmac_v4 = 0, tmac_z = 0, umac_z = 0;
  double zc_tmax = 0, zc_tavg = 0;  // summed over the waves' D_FG / D_FB launches
  // D_FG and D_FB pieces on the tensor cores (HFX_ZJOBS=0 keeps them in FP64)
  const char *zenv = std::getenv("HFX_ZJOBS");
  const bool zjobs = split && !(zenv && zenv[0] == '0');
  CK(cudaEventRecord(ctx->ev[1], st));
  // ---- contraction waves
  const size_t budget = scratch_budget_doubles();
  int64_t nwaves = 0;
  size_t peak = 0;
  {
    const size_t nit_all = ctx->items.size();
    // item ranges of the central atoms this context owns (all without a shard)
    std::vector<std::pair<size_t, size_t>> ranges;
    for (size_t q = 0; q < nit_all;) {
      size_t e = q;
      while (e < nit_all && ctx->items[e].a == ctx->items[q].a) ++e;
      const bool mine = ctx->owner.empty() || ctx->owner[ctx->items[q].a] == ctx->rank;
      if (mine) {
        if (!ranges.empty() && ranges.back().second == q) ranges.back().second = e;
        else ranges.push_back({q, e});
      }
      q = e;
    }
    std::vector<int64_t> offs4;
    for (const auto &rg : ranges) {
    const size_t nit = rg.second;
    size_t w0 = rg.first;
    while (w0 < nit) {
      size_t w1 = w0;
      size_t used = 0;
      offs4.clear();
      std::vector<int64_t> yo, po, to, qo, y2o;
      while (w1 < nit) {
        const WorkItem &it = ctx->items[w1];
        const int64_t pA = ctx->nabf[it.a], na = ctx->nao[it.a], nb = ctx->nao[it.b];
        // every region starts on a 256-byte boundary (bulk copies read Y2)
        auto pad = [](int64_t x) { return (x + 31) / 32 * 32; };
        // FP64 Y: not read at all with the tensor D_FG / D_FB products and mirror
        // pieces (P of the D_AB piece is built from the f32 pairs)
        const bool y64 = !(split && zjobs && ctx->sym);
        const int64_t ysz = y64 ? pad(pA * nb * ctx->aotot[it.b]) : 0;
        const int64_t psz = (it.dab >= 0 && !split) ? pad(pA * na * ctx->aotot[it.b]) : 0;
        // T3 only for the D_AG piece without mirrors; Q only for the FP64 D_FB piece
        const int64_t tsz = ctx->sym ? 0 : pad((int64_t)it.nG * pA * na * nb);
        const int64_t qsz = zjobs ? 0 : pad((int64_t)it.nF * pA * na * nb);
        // Y as f32 pairs in 16-column blocks (D_FG / D_FB products and P)
        const int64_t pssz = split ? pad(pA * nb * ctx->ktotZ_h[it.b]) : 0;
        const size_t need = (size_t)(ysz + psz + tsz + qsz + pssz);
        if (w1 > w0 && used + need > budget) break;
        yo.push_back((int64_t)used);
        po.push_back((int64_t)used + ysz);
        to.push_back((int64_t)used + ysz + psz);
        qo.push_back((int64_t)used + ysz + psz + tsz);
        y2o.push_back((int64_t)used + ysz + psz + tsz + qsz);
        used += need;
        ++w1;
      }
      const size_t nw = w1 - w0;
      offs4.insert(offs4.end(), yo.begin(), yo.end());
      offs4.insert(offs4.end(), po.begin(), po.end());
      offs4.insert(offs4.end(), to.begin(), to.end());
      offs4.insert(offs4.end(), qo.begin(), qo.end());
      offs4.insert(offs4.end(), y2o.begin(), y2o.end());
      CK(ctx->d_scratch.reserve(std::max<size_t>(used, 1)));
      CK(ctx->d_waveoffs.reserve(offs4.size()));
      CK(cudaMemcpyAsync(ctx->d_waveoffs.p, offs4.data(), sizeof(int64_t) * offs4.size(),
                         cudaMemcpyHostToDevice, st));
      peak = std::max(peak, used);
      ContractArgs c{};
      c.items = ctx->d_items.p;
      c.w0 = (int64_t)w0;
      c.w1 = (int64_t)w1;
      c.wg_base = ctx->items[w0].wg_off;
      c.wf_base = ctx->items[w0].wf_off;
      const int64_t wg_end = (w1 < nit_all) ? ctx->items[w1].wg_off : ctx->nwg;
      const int64_t wf_end = (w1 < nit_all) ? ctx->items[w1].wf_off : ctx->nwf;
      c.nwg = wg_end - c.wg_base;
      c.nwf = wf_end - c.wf_base;
      c.nbr = ctx->d_nbr.p;
      c.nao = ctx->d_nao.p;
      c.nabf = ctx->d_nabf.p;
      c.ncol = ctx->d_ncol.p;
      c.C = DevBlocks{ctx->K[0].data.p, ctx->K[0].d_offs.p, ctx->K[0].maxabs.p};
      c.V = DevBlocks{ctx->K[1].data.p, ctx->K[1].d_offs.p, ctx->K[1].maxabs.p};
      c.D = DevBlocks{ctx->K[2].data.p, ctx->K[2].d_offs.p, ctx->K[2].maxabs.p};
      c.dhash = DevHash{ctx->d_dhkeys.p, ctx->d_dhvals.p, ctx->dmask};
      c.shash = DevHash{ctx->d_shkeys.p, ctx->d_shvals.p, ctx->smask};
      c.masks = ctx->d_masks.p;
      c.wg_flags = ctx->d_wg.p;
      c.wf_flags = ctx->d_wf.p;
      c.scratch = ctx->d_scratch.p;
      c.y_off = ctx->d_waveoffs.p;
      c.p_off = ctx->d_waveoffs.p + nw;
      c.t3_off = ctx->d_waveoffs.p + 2 * nw;
      c.q_off = ctx->d_waveoffs.p + 3 * nw;
      c.acc = ctx->d_acc.p;
      c.macs = ctx->d_counters.p + 8;
      c.err = ctx->d_err.p;
      c.sym = ctx->sym ? 1 : 0;
      int nl = 0;
      int zc_ctas[2] = {0, 0};  // CTAs of the small-class and the other D_FG / D_FB launch
      SplitWave SW{};
      if (split) {
        // per-wave split metadata
        std::vector<int64_t> prow(nw + 1, 0), psb(nw, -1), ycand(nw + 1, 0), v4cand(nw + 1, 0),
            pgcand(nw + 1, 0);
        int64_t ps_elems = 0, v4max = 0;
        for (size_t q = 0; q < nw; ++q) {
          const WorkItem &it = ctx->items[w0 + q];
          const int64_t ntv = (ctx->nabf[it.a] + 63) / 64;
          (void)ntv;
          const bool has = it.dab >= 0 && !(ctx->sym && it.role == 2);
          const int64_t ntp = (ctx->aotot[it.b] + 63) / 64, mt4 = (ctx->aotot[it.a] + 127) / 128;
          prow[q + 1] = prow[q] + (has ? ntp * 64 : 0);
          pgcand[q + 1] = pgcand[q] + (has ? it.nG : 0);
          v4cand[q + 1] = v4cand[q] + (has ? mt4 * ntp : 0);
          if (has) {
            psb[q] = ps_elems;
            ps_elems += ntp * ctx->kt4[it.a] * nslices * 64 * 32;
            v4max += mt4 * ntp * ((ctx->kt4[it.a] + 19) / 20);
          }
        }
        // Y candidates with the items grouped by atom B (stable), so that Y jobs
        // running side by side share C_B digit tiles in L2
        std::vector<int64_t> yperm(nw);
        for (size_t q = 0; q < nw; ++q) yperm[q] = (int64_t)q;
        std::stable_sort(yperm.begin(), yperm.end(), [&](int64_t x, int64_t y) {
          return ctx->items[w0 + x].b < ctx->items[w0 + y].b;
        });
        for (size_t k = 0; k < nw; ++k) {
          const WorkItem &it = ctx->items[w0 + yperm[k]];
          const int64_t ntv = (ctx->nabf[it.a] + 63) / 64;
          const int64_t mty = ((int64_t)ctx->nao[it.b] * ctx->aotot[it.b] + 127) / 128;
          ycand[k + 1] = ycand[k] + mty * ntv;
        }
        std::vector<int64_t> wm;
        wm.insert(wm.end(), prow.begin(), prow.end());
        wm.insert(wm.end(), psb.begin(), psb.end());
        wm.insert(wm.end(), ycand.begin(), ycand.end());
        wm.insert(wm.end(), v4cand.begin(), v4cand.end());
        wm.insert(wm.end(), yperm.begin(), yperm.end());
        wm.insert(wm.end(), pgcand.begin(), pgcand.end());
        CK(ctx->d_wave_split.reserve(wm.size()));
        CK(cudaMemcpyAsync(ctx->d_wave_split.p, wm.data(), sizeof(int64_t) * wm.size(),
                           cudaMemcpyHostToDevice, st));
        CK(ctx->d_ps.reserve(std::max<int64_t>(ps_elems, 1)));
        CK(ctx->d_ps_e.reserve(std::max<int64_t>(prow[nw], 1)));
        CK(ctx->d_jobs.reserve(std::max<int64_t>(ycand[nw], 1)));
        CK(ctx->d_jobs4.reserve(std::max<int64_t>(v4max, 1)));
        CK(cudaMemsetAsync(ctx->d_njobs.p, 0, 4 * sizeof(int), st));
        CK(cudaMemsetAsync(ctx->d_tmacs.p, 0, 4 * sizeof(unsigned long long), st));
        SW.w0 = (int64_t)w0;
        SW.nw = (int32_t)nw;
        SW.scratch = ctx->d_scratch.p;
        SW.y_off = c.y_off;
        SW.p_off = c.p_off;
        SW.p_rowpre = ctx->d_wave_split.p;
        SW.ps_base = ctx->d_wave_split.p + (nw + 1);
        SW.y_candpre = ctx->d_wave_split.p + (nw + 1) + nw;
        SW.v4_candpre = ctx->d_wave_split.p + 2 * (nw + 1) + nw;
        SW.y_perm = ctx->d_wave_split.p + 3 * (nw + 1) + nw;
        SW.pg_candpre = ctx->d_wave_split.p + 3 * (nw + 1) + 2 * nw;
        SW.h_pgcand = pgcand[nw];
        SW.y2_off = ctx->d_waveoffs.p + 4 * nw;
        SW.y2_on = 1;
        SW.y64_mode = (zjobs && ctx->sym) ? 2 : 1;
        SW.ps = ctx->d_ps.p;
        SW.ps_e = ctx->d_ps_e.p;
        SW.jobs = ctx->d_jobs.p;
        SW.jobs4 = ctx->d_jobs4.p;
        SW.njobs = ctx->d_njobs.p;
        SW.tmacs = ctx->d_tmacs.p;
        SW.h_ycand = ycand[nw];
        SW.h_v4cand = v4cand[nw];
        SW.h_prows = prow[nw];
        SW.h_v4jobs_max = v4max;
        CK(cudaEventRecord(ctx->sev[0], st));
        CK(split_wave(SS, SW, nslices, 0, st));
        CK(cudaEventRecord(ctx->sev[1], st));
        ctx->launches += 2;
        // Y and the D_AB piece run on the tensor cores; the D_FG and D_FB pieces
        // too when the Z-job form is selected (HFX_ZJOBS=1)
        c.skip = zjobs ? (1u | 4u | 8u | 32u | 64u) : (1u | 64u);
        // P of the D_AB piece is computed and sliced in phase 1; the D-stage is
        // left with T3, needed only without mirror pieces
        c.no_p = 1;
        if (ctx->sym) c.skip |= 2u;
      }
      CK(launch_contract_fp64(c, st, ctx->kev, &nl));
      ctx->launches += nl;
      if (split) {
        CK(cudaEventRecord(ctx->sev[2], st));
        CK(split_wave(SS, SW, nslices, 1, st));
        CK(cudaEventRecord(ctx->sev[3], st));
        ctx->launches += (SW.h_pgcand > 0) + (SW.h_v4cand > 0) + 1;
      }
      if (split && zjobs) {
        // D_FG and D_FB pieces: count jobs and entries and histogram their cost
        // keys, size the lists, place the jobs longest first (Algorithm 6's
        // order), plan and run
        constexpr int NKEYS = 512, NCOST = 256;  // size class x cost
        CK(ctx->d_zckeys.reserve(NKEYS));
        CK(ctx->d_ctans.reserve(2 * std::max(ctx->nsm, 1)));
        CK(cudaMemsetAsync(ctx->d_zckeys.p, 0, NKEYS * sizeof(int), st));
        SW.zc_keys = ctx->d_zckeys.p;
        SW.cta_ns = ctx->d_ctans.p;
        CK(cudaEventRecord(ctx->kev[8], st));
        CK(split_zc_plan(SS, SW, 0, st));
        int nz[2] = {0, 0};
        std::vector<int> hist(NKEYS, 0);
        CK(cudaMemcpyAsync(nz, ctx->d_njobs.p + 2, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(hist.data(), ctx->d_zckeys.p, NKEYS * sizeof(int),
                           cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        // the small class's range first, each class longest first
        int nsmall = 0;
        for (int key = 0; key < NCOST; ++key) nsmall += hist[key];
        {
          int off = 0;
          for (int cls = 0; cls < 2; ++cls)
            for (int key = cls * NCOST + NCOST - 1; key >= cls * NCOST; --key) {
              const int c = hist[key];
              hist[key] = off;
              off += c;
            }
        }
        CK(cudaMemcpyAsync(ctx->d_zckeys.p, hist.data(), NKEYS * sizeof(int),
                           cudaMemcpyHostToDevice, st));
        CK(ctx->d_zcjobs.reserve(std::max(nz[0], 1)));
        CK(ctx->d_zcents.reserve(std::max(nz[1], 1)));
        CK(cudaMemsetAsync(ctx->d_njobs.p + 2, 0, 2 * sizeof(int), st));
        SW.zc_jobs = ctx->d_zcjobs.p;
        SW.zc_ents = ctx->d_zcents.p;
        SW.h_zc_jobs = nz[0];
        CK(split_zc_plan(SS, SW, 1, st));
        CK(split_zc_run(SS, SW, nslices, ctx->zc_shape, ctx->nsm, nsmall, st));
        CK(cudaEventRecord(ctx->kev[9], st));
        ctx->launches += 2 * (nw > 0) + (nsmall > 0) + (nz[0] > nsmall);
        zc_ctas[0] = (int)std::min<int64_t>(nsmall, ctx->nsm);
        zc_ctas[1] = (int)std::min<int64_t>(nz[0] - nsmall, ctx->nsm);
      }
      // the host offsets vector is reused next wave: order the copy first
      CK(cudaStreamSynchronize(st));
      for (int q = 0; q < 7; ++q) {
        float ms = 0;
        cudaEventElapsedTime(&ms, ctx->kev[q], ctx->kev[q + 1]);
        kms[1 + q] += ms;
      }
      if (split) {
        float ms = 0;
        cudaEventElapsedTime(&ms, ctx->sev[0], ctx->sev[1]);
        kms[1] += ms;
        cudaEventElapsedTime(&ms, ctx->sev[2], ctx->sev[3]);
        kms[7] += ms;
        if (zjobs) {
          cudaEventElapsedTime(&ms, ctx->kev[8], ctx->kev[9]);
          kms[4] += ms;
        }
        unsigned long long tm[4] = {0, 0, 0, 0};
        CK(cudaMemcpyAsync(tm, ctx->d_tmacs.p, sizeof(tm), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        tmac_y += (double)tm[0];
        tmac_v4 += (double)tm[1];
        tmac_z += (double)tm[2];
        umac_z += (double)tm[3];
        for (int l = 0; l < 2; ++l) {
          if (zc_ctas[l] <= 0) continue;
          // load balance of each launch: largest and mean CTA busy time
          std::vector<long long> ns(zc_ctas[l]);
          CK(cudaMemcpyAsync(ns.data(), ctx->d_ctans.p + l * ctx->nsm,
                             sizeof(long long) * zc_ctas[l], cudaMemcpyDeviceToHost, st));
          CK(cudaStreamSynchronize(st));
          double mx = 0, sum = 0;
          for (long long v : ns) {
            mx = std::max(mx, (double)v);
            sum += (double)v;
          }
          zc_tmax += mx;
          zc_tavg += sum / zc_ctas[l];
        }
      }
      ++nwaves;
      w0 = w1;
    }
    }
  }
  CK(cudaEventRecord(ctx->ev[2], st));
  // ---- finalize
  const int64_t nelem = ctx->sig_offs[nsig];
  CK(ctx->d_sigma.reserve(nelem));
  CK(ctx->d_partials.reserve(nsig));
  CK(launch_finalize(ctx->d_acc.p, nelem, ctx->d_sigma.p, ctx->d_skeys.p, ctx->d_soffs.p, nsig,
                     DevBlocks{ctx->K[2].data.p, ctx->K[2].d_offs.p, ctx->K[2].maxabs.p},
                     DevHash{ctx->d_dhkeys.p, ctx->d_dhvals.p, ctx->dmask}, ctx->d_partials.p,
                     ctx->d_ex.p, st));
  ctx->launches += (nelem > 0) + (nsig > 0) + 1;
  CK(cudaEventRecord(ctx->ev[3], st));
  double ex = 0.0;
  CK(cudaMemcpyAsync(&ex, ctx->d_ex.p, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&herr, ctx->d_err.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  unsigned long long kmacs[7] = {0};
  CK(cudaMemcpyAsync(kmacs, ctx->d_counters.p + 8, sizeof(kmacs), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (herr) return fail(ctx, HFX_E_CUDA, "contraction kernels reported error " + std::to_string(herr));
  float ms01 = 0, ms12 = 0, ms23 = 0, ms03 = 0;
  cudaEventElapsedTime(&ms01, ctx->ev[0], ctx->ev[1]);
  cudaEventElapsedTime(&ms12, ctx->ev[1], ctx->ev[2]);
  cudaEventElapsedTime(&ms23, ctx->ev[2], ctx->ev[3]);
  cudaEventElapsedTime(&ms03, ctx->ev[0], ctx->ev[3]);
  hfx_stats_v1 &S = ctx->stats;
  S = hfx_stats_v1{};
  S.version = 1;
  S.prec = (int32_t)prec;
  S.theta = theta;
  S.n_sigma_blocks = nsig;
  S.n_work_items = (int64_t)ctx->items.size();
  S.n_active_abg = (int64_t)counters[4];
  for (int v = 0; v < 4; ++v) S.survivors[v] = (int64_t)counters[v];
  S.canonical_flops = 2.0 * (double)counters[5];
  for (int v = 0; v < 4; ++v) S.canonical_flops_piece[v] = 2.0 * (double)counters[16 + v];
  S.canonical_flops_y = 2.0 * (double)counters[20];
  S.eps_eri = ctx->eps_eri;
  S.n_eri_removed = (int64_t)counters[21];
  double macs = 0;
  for (int q = 0; q < 7; ++q) macs += (double)kmacs[q];
  S.executed_flops = 2.0 * macs;
  // stats kernel order: screen, Y, D-stage, Q, D_FG, D_AG, D_FB, D_AB
  // (kmacs / kms[1..7] are in launch order: Y, D-stage, Q, D_FG, D_AG, D_FB, D_AB)
  for (int q = 0; q < 8; ++q) S.kernel_ms[q] = kms[q];
  S.kernel_flops[0] = 0.0;
  for (int q = 0; q < 7; ++q) S.kernel_flops[1 + q] = 2.0 * (double)kmacs[q];
  S.n_launches = ctx->launches;
  S.mirror = ctx->sym ? 1 : 0;
  S.nslices = split ? nslices : 0;
  if (split) {
    const double pairs = (double)nslices * (nslices + 1) / 2;
    S.kernel_flops[1] += 2.0 * tmac_y;
    S.kernel_flops[7] += 2.0 * tmac_v4;
    S.executed_flops += 2.0 * (tmac_y + tmac_v4);
    S.kernel_tensor_flops[1] = 2.0 * tmac_y * pairs;
    S.kernel_tensor_flops[7] = 2.0 * tmac_v4 * pairs;
    S.kernel_flops[4] += 2.0 * tmac_z;
    S.executed_flops += 2.0 * tmac_z;
    S.kernel_tensor_flops[4] = 2.0 * tmac_z * pairs;
    // FP64-equivalent work of the tensor products without padding or zero
    // tiles: the Y product's canonical count, the D_FG / D_FB products' count
    // from the job plan
    S.kernel_unpadded_flops[1] = S.canonical_flops_y;
    S.kernel_unpadded_flops[4] = 2.0 * umac_z;
    S.zc_dt_max_over_avg = zc_tavg > 0 ? zc_tmax / zc_tavg : 0.0;
  }
  S.ms_screen = ms01;
  S.ms_contract = ms12;
  S.ms_reduce = ms23;
  S.ms_total = ms03;
  S.n_waves = nwaves;
  S.scratch_bytes = (int64_t)(peak * sizeof(double));
  ctx->ex = ex;
  ctx->results_valid = true;
  if (ex_out) *ex_out = ex;
  return HFX_OK;
}

}  // extern "C"

namespace {

// Copy one kind of a cell's blocks into the merged system m, atoms offset
// by first (blocks already there are replaced).
hfx_status copy_cell_kind(hfx_ctx *m, hfx_ctx *ctx, int k, int32_t first) {
  // packing here must not hide from the cell's own next build that its
  // blocks changed since its last one: keep the kind's dirty flag
  const bool was_dirty = ctx->K[k].dirty;
  hfx_status s = pack_kind(ctx, k);
  ctx->K[k].dirty = was_dirty;
  if (s != HFX_OK) return s;
  if (ctx->stream && cudaStreamSynchronize(ctx->stream) != cudaSuccess)
    return fail(ctx, HFX_E_CUDA, "batch: stream synchronisation failed");
  const Kind &K = ctx->K[k];
  const int64_t nblk = (int64_t)K.keys.size();
  if (nblk == 0) return HFX_OK;
  std::vector<int32_t> keys(5 * nblk);
  for (int64_t e = 0; e < nblk; ++e) {
    hk_unpack(K.keys[e], &keys[5 * e]);
    keys[5 * e] += first;
    keys[5 * e + 1] += first;
  }
  s = hfx_set_many(m, K.name, nblk, keys.data(), K.data.p, K.offs.data(), 1);
  if (s != HFX_OK) fail(ctx, s, std::string("batch: ") + m->err);
  return s;
}

// The cells of a batch as one system: cell c's atoms follow those of cells
// 0 .. c-1, its blocks keep their keys with both atoms offset, and no block
// joins two cells, so the merged build's terms are exactly the union of the
// cells' terms.  The packed device data of each cell is copied as it is.
hfx_status merge_cells(hfx_ctx *const *cells, int32_t ncells, const double *thetas,
                       std::vector<int32_t> &first, hfx_ctx **out) {
  first.assign(ncells + 1, 0);
  for (int32_t c = 0; c < ncells; ++c) first[c + 1] = first[c] + cells[c]->natoms;
  const int32_t natoms = first[ncells];
  if (natoms >= (1 << 20)) return fail(cells[0], HFX_E_SHAPE, "batch: more than 2^20 atoms");
  std::vector<int32_t> nao(natoms), nabf(natoms), species(natoms);
  for (int32_t c = 0; c < ncells; ++c)
    for (int32_t a = 0; a < cells[c]->natoms; ++a) {
      nao[first[c] + a] = cells[c]->nao[a];
      nabf[first[c] + a] = cells[c]->nabf[a];
    }
  for (int32_t a = 0; a < natoms; ++a) species[a] = a;
  hfx_ctx *m = nullptr;
  hfx_status s = hfx_create(nullptr, natoms, nullptr, species.data(), natoms, nao.data(),
                            nabf.data(), cells[0]->stream, &m);
  if (s != HFX_OK) return fail(cells[0], s, "batch: cannot create the merged system");
  for (int32_t c = 0; c < ncells && s == HFX_OK; ++c)
    for (int k = 0; k < 3 && s == HFX_OK; ++k) s = copy_cell_kind(m, cells[c], k, first[c]);
  if (s != HFX_OK) {
    hfx_destroy(m);
    return s;
  }
  *out = m;
  return HFX_OK;
}

}  // namespace

extern "C" {

hfx_status hfx_build_batch(hfx_ctx **cells, int32_t ncells, const double *thetas, hfx_prec prec,
                           int32_t nslices, double *ex_out) {
  if (ncells < 0 || (ncells > 0 && (!cells || !thetas))) return HFX_E_ARG;
  if (ncells == 0) return HFX_OK;
  for (int32_t c = 0; c < ncells; ++c) {
    if (!cells[c]) return HFX_E_ARG;
    if (!(thetas[c] >= 0.0) || !std::isfinite(thetas[c]))
      return fail(cells[c], HFX_E_ARG, "batch: theta must be >= 0");
    for (int32_t d = 0; d < c; ++d)
      if (cells[d] == cells[c]) return fail(cells[c], HFX_E_ARG, "batch: a cell appears twice");
    if (cells[c]->eps_eri != cells[0]->eps_eri)
      return fail(cells[c], HFX_E_ARG, "batch: the cells' ERI screen thresholds differ");
    cells[c]->results_valid = false;
  }
  // the merged system of the last batch of the same cells is reused when no
  // cell's C or V blocks changed and no D key set changed: its plan and
  // sliced operands stay valid, and changed D values are copied in again
  std::vector<uint64_t> ids(ncells);
  std::vector<std::array<uint64_t, 3>> gens(ncells), kgens(ncells);
  for (int32_t c = 0; c < ncells; ++c) {
    ids[c] = cells[c]->id;
    for (int k = 0; k < 3; ++k) {
      gens[c][k] = cells[c]->gen[k];
      kgens[c][k] = cells[c]->kgen[k];
    }
  }
  BatchCache *bc = cells[0]->batch.get();
  bool reuse = bc && bc->ids == ids;
  for (int32_t c = 0; reuse && c < ncells; ++c)
    reuse = bc->gens[c][0] == gens[c][0] && bc->gens[c][1] == gens[c][1] &&
            bc->kgens[c][2] == kgens[c][2];
  hfx_status s = HFX_OK;
  if (reuse) {
    for (int32_t c = 0; c < ncells && s == HFX_OK; ++c)
      if (bc->gens[c][2] != gens[c][2]) s = copy_cell_kind(bc->merged, cells[c], 2, bc->first[c]);
  } else {
    cells[0]->batch.reset();
    std::vector<int32_t> first;
    hfx_ctx *m0 = nullptr;
    s = merge_cells(cells, ncells, thetas, first, &m0);
    if (s == HFX_OK) {
      cells[0]->batch.reset(new BatchCache());
      bc = cells[0]->batch.get();
      bc->ids = ids;
      bc->first = first;
      bc->merged = m0;
    }
  }
  if (s != HFX_OK) {
    cells[0]->batch.reset();
    return s;
  }
  hfx_ctx *m = bc->merged;
  const std::vector<int32_t> &first = bc->first;
  m->theta_atom.resize(first[ncells]);
  for (int32_t c = 0; c < ncells; ++c)
    for (int32_t a = first[c]; a < first[c + 1]; ++a) m->theta_atom[a] = thetas[c];
  m->eps_eri = cells[0]->eps_eri;
  m->results_valid = false;
  s = hfx_build(m, 0.0, prec, nslices, nullptr);
  if (s != HFX_OK) {
    for (int32_t c = 0; c < ncells; ++c) fail(cells[c], s, "batch: " + m->err);
    cells[0]->batch.reset();
    return s;
  }
  bc->gens = gens;
  bc->kgens = kgens;
  // Sigma, its fixed-point words and E_X of each cell from the merged result:
  // cell c's keys are the contiguous range with first atom in [first[c],
  // first[c + 1]); E_X reduces that range's per-block partials exactly as a
  // build of the cell alone does
  hfx_ctx *ctx = nullptr;
  auto fail_all = [&](const char *what, cudaError_t e) {
    for (int32_t c = 0; c < ncells; ++c)
      fail(cells[c], HFX_E_CUDA, std::string("batch: ") + what + ": " + cudaGetErrorString(e));
    cells[0]->batch.reset();
    return HFX_E_CUDA;
  };
  cudaStream_t st = m->stream;
  cudaError_t e = m->d_ex_cells.reserve(ncells);
  if (e != cudaSuccess) return fail_all("cudaMalloc", e);
  std::vector<int64_t> k0(ncells), k1(ncells);
  for (int32_t c = 0; c < ncells; ++c) {
    k0[c] = std::lower_bound(m->sig_keys.begin(), m->sig_keys.end(),
                             (uint64_t)first[c] << 44) - m->sig_keys.begin();
    k1[c] = std::lower_bound(m->sig_keys.begin(), m->sig_keys.end(),
                             (uint64_t)first[c + 1] << 44) - m->sig_keys.begin();
    e = launch_ex_reduce(m->d_partials.p + k0[c], k1[c] - k0[c], m->d_ex_cells.p + c, st);
    if (e != cudaSuccess) return fail_all("E_X reduction", e);
  }
  std::vector<double> exs(ncells);
  e = cudaMemcpyAsync(exs.data(), m->d_ex_cells.p, sizeof(double) * ncells,
                      cudaMemcpyDeviceToHost, st);
  for (int32_t c = 0; c < ncells && e == cudaSuccess; ++c) {
    ctx = cells[c];
    const int64_t nk = k1[c] - k0[c];
    const int64_t e0 = m->sig_offs[k0[c]], ne = m->sig_offs[k1[c]] - e0;
    ctx->sig_keys.resize(nk);
    ctx->sig_offs.assign(nk + 1, 0);
    for (int64_t q = 0; q < nk; ++q) {
      int32_t kk[5];
      hk_unpack(m->sig_keys[k0[c] + q], kk);
      ctx->sig_keys[q] = hk_pack(kk[0] - first[c], kk[1] - first[c], kk[2], kk[3], kk[4]);
      ctx->sig_offs[q + 1] = m->sig_offs[k0[c] + q + 1] - e0;
    }
    e = ctx->d_sigma.reserve(std::max<int64_t>(ne, 1));
    if (e == cudaSuccess) e = ctx->d_acc.reserve(2 * std::max<int64_t>(ne, 1));
    if (e == cudaSuccess && ne > 0)
      e = cudaMemcpyAsync(ctx->d_sigma.p, m->d_sigma.p + e0, sizeof(double) * ne,
                          cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && ne > 0)
      e = cudaMemcpyAsync(ctx->d_acc.p, m->d_acc.p + 2 * e0, sizeof(unsigned long long) * 2 * ne,
                          cudaMemcpyDeviceToDevice, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail_all("copying the cells' results", e);
  for (int32_t c = 0; c < ncells; ++c) {
    ctx = cells[c];
    ctx->ex = exs[c];
    ctx->stats = m->stats;  // batch-wide counts and times
    ctx->results_valid = true;
    ctx->from_batch = true;
    if (ex_out) ex_out[c] = exs[c];
  }
  return HFX_OK;
}

hfx_status hfx_set_eri_screen(hfx_ctx *ctx, double eps_eri) {
  if (!ctx) return HFX_E_ARG;
  if (std::isnan(eps_eri) || std::isinf(eps_eri))
    return fail(ctx, HFX_E_ARG, "eps_eri must be finite (negative turns the screen off)");
  ctx->eps_eri = eps_eri < 0.0 ? -1.0 : eps_eri;
  ctx->results_valid = false;
  return HFX_OK;
}

hfx_status hfx_set_shard(hfx_ctx *ctx, const int32_t *owner, int32_t rank) {
  if (!ctx) return HFX_E_ARG;
  if (!owner) {
    ctx->owner.clear();
    ctx->rank = 0;
    ctx->results_valid = false;
    return HFX_OK;
  }
  if (rank < 0) return fail(ctx, HFX_E_ARG, "rank must be >= 0");
  for (int a = 0; a < ctx->natoms; ++a)
    if (owner[a] < 0) return fail(ctx, HFX_E_ARG, "owner ranks must be >= 0");
  ctx->owner.assign(owner, owner + ctx->natoms);
  ctx->rank = rank;
  ctx->results_valid = false;
  return HFX_OK;
}

hfx_status hfx_get_H_fixed(const hfx_ctx *ctx, int64_t *words, int on_device) {
  if (!ctx || !words) return HFX_E_ARG;
  if (!ctx->results_valid) return HFX_E_STATE;
  const int64_t n = ctx->sig_offs.empty() ? 0 : ctx->sig_offs.back();
  if (n == 0) return HFX_OK;
  if (cudaMemcpyAsync(words, ctx->d_acc.p, sizeof(int64_t) * 2 * n,
                      on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                      ctx->stream) != cudaSuccess ||
      cudaStreamSynchronize(ctx->stream) != cudaSuccess)
    return HFX_E_CUDA;
  return HFX_OK;
}

hfx_status hfx_set_H_fixed(hfx_ctx *ctx, const int64_t *words, int on_device, double *ex_out) {
  if (!ctx || !words) return HFX_E_ARG;
  if (!ctx->results_valid) return fail(ctx, HFX_E_STATE, "no build whose key set to use");
  if (ctx->from_batch)
    return fail(ctx, HFX_E_STATE, "results of a batch build: build the cell alone to shard it");
  cudaStream_t st = ctx->stream;
  const int64_t nsig = (int64_t)ctx->sig_keys.size();
  const int64_t nelem = ctx->sig_offs.empty() ? 0 : ctx->sig_offs.back();
  if (nelem > 0)
    CK(cudaMemcpyAsync(ctx->d_acc.p, words, sizeof(int64_t) * 2 * nelem,
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  CK(launch_finalize(ctx->d_acc.p, nelem, ctx->d_sigma.p, ctx->d_skeys.p, ctx->d_soffs.p, nsig,
                     DevBlocks{ctx->K[2].data.p, ctx->K[2].d_offs.p, ctx->K[2].maxabs.p},
                     DevHash{ctx->d_dhkeys.p, ctx->d_dhvals.p, ctx->dmask}, ctx->d_partials.p,
                     ctx->d_ex.p, st));
  double ex = 0.0;
  CK(cudaMemcpyAsync(&ex, ctx->d_ex.p, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  ctx->ex = ex;
  if (ex_out) *ex_out = ex;
  return HFX_OK;
}

hfx_status hfx_H_count(const hfx_ctx *ctx, int64_t *nblk) {
  if (!ctx || !nblk) return HFX_E_ARG;
  if (!ctx->results_valid) return HFX_E_STATE;
  *nblk = (int64_t)ctx->sig_keys.size();
  return HFX_OK;
}

hfx_status hfx_H_keys(const hfx_ctx *ctx, int32_t *keys) {
  if (!ctx || !keys) return HFX_E_ARG;
  if (!ctx->results_valid) return HFX_E_STATE;
  for (size_t e = 0; e < ctx->sig_keys.size(); ++e) hk_unpack(ctx->sig_keys[e], keys + 5 * e);
  return HFX_OK;
}

hfx_status hfx_H_offsets(const hfx_ctx *ctx, int64_t *offs) {
  if (!ctx || !offs) return HFX_E_ARG;
  if (!ctx->results_valid) return HFX_E_STATE;
  std::memcpy(offs, ctx->sig_offs.data(), sizeof(int64_t) * ctx->sig_offs.size());
  return HFX_OK;
}

hfx_status hfx_get_H(const hfx_ctx *ctx, int32_t i, int32_t j, const int32_t n[3], double *out) {
  if (!ctx || !n || !out) return HFX_E_ARG;
  if (!ctx->results_valid) return HFX_E_STATE;
  const uint64_t k = hk_pack(i, j, n[0], n[1], n[2]);
  auto it = std::lower_bound(ctx->sig_keys.begin(), ctx->sig_keys.end(), k);
  if (it == ctx->sig_keys.end() || *it != k) return HFX_E_NOTFOUND;
  const size_t e = (size_t)(it - ctx->sig_keys.begin());
  const int64_t len = ctx->sig_offs[e + 1] - ctx->sig_offs[e];
  if (cudaMemcpyAsync(out, ctx->d_sigma.p + ctx->sig_offs[e], sizeof(double) * len,
                      cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
      cudaStreamSynchronize(ctx->stream) != cudaSuccess)
    return HFX_E_CUDA;
  return HFX_OK;
}

hfx_status hfx_get_H_all(const hfx_ctx *ctx, double *out, int on_device) {
  if (!ctx || !out) return HFX_E_ARG;
  if (!ctx->results_valid) return HFX_E_STATE;
  const int64_t n = ctx->sig_offs.empty() ? 0 : ctx->sig_offs.back();
  if (n == 0) return HFX_OK;
  if (cudaMemcpyAsync(out, ctx->d_sigma.p, sizeof(double) * n,
                      on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                      ctx->stream) != cudaSuccess ||
      cudaStreamSynchronize(ctx->stream) != cudaSuccess)
    return HFX_E_CUDA;
  return HFX_OK;
}

hfx_status hfx_grad(hfx_ctx *ctx, double *dC, double *dV) {
  if (!ctx) return HFX_E_ARG;
  if (!ctx->results_valid) return fail(ctx, HFX_E_STATE, "no build to differentiate");
  if (ctx->from_batch)
    return fail(ctx, HFX_E_STATE, "results of a batch build: build the cell alone to differentiate");
  cudaStream_t st = ctx->stream;
  const int64_t nC = ctx->K[0].offs.back(), nV = ctx->K[1].offs.back();
  DevBuf<unsigned long long> dcacc;
  DevBuf<double> dcout, dvout;
  CK(dcacc.reserve(2 * nC));
  CK(dcout.reserve(nC));
  CK(dvout.reserve(nV));
  CK(cudaMemsetAsync(dcacc.p, 0, sizeof(unsigned long long) * 2 * (nC ? nC : 1), st));
  CK(cudaMemsetAsync(dvout.p, 0, sizeof(double) * (nV ? nV : 1), st));
  CK(cudaMemsetAsync(ctx->d_err.p, 0, sizeof(unsigned), st));
  CK(cudaMemsetAsync(ctx->d_counters.p + 8, 0, sizeof(unsigned long long) * 7, st));
  // waves over the pairs: Y and R per pair
  const size_t budget = scratch_budget_doubles();
  const size_t nit = ctx->items.size();
  size_t w0 = 0;
  while (w0 < nit) {
    size_t w1 = w0, used = 0;
    std::vector<int64_t> yo, ro;
    while (w1 < nit) {
      const WorkItem &it = ctx->items[w1];
      const int64_t ysz = (int64_t)ctx->nabf[it.a] * ctx->nao[it.b] * ctx->aotot[it.b];
      if (w1 > w0 && used + 2 * ysz > budget) break;
      yo.push_back((int64_t)used);
      ro.push_back((int64_t)used + ysz);
      used += 2 * ysz;
      ++w1;
    }
    const size_t nw = w1 - w0;
    std::vector<int64_t> offs(yo);
    offs.insert(offs.end(), ro.begin(), ro.end());
    CK(ctx->d_scratch.reserve(std::max<size_t>(used, 1)));
    CK(ctx->d_waveoffs.reserve(offs.size()));
    CK(cudaMemcpyAsync(ctx->d_waveoffs.p, offs.data(), sizeof(int64_t) * offs.size(),
                       cudaMemcpyHostToDevice, st));
    ContractArgs c{};
    c.items = ctx->d_items.p;
    c.w0 = (int64_t)w0;
    c.w1 = (int64_t)w1;
    c.wg_base = ctx->items[w0].wg_off;
    c.wf_base = ctx->items[w0].wf_off;
    c.nwg = ((w1 < nit) ? ctx->items[w1].wg_off : ctx->nwg) - c.wg_base;
    c.nwf = ((w1 < nit) ? ctx->items[w1].wf_off : ctx->nwf) - c.wf_base;
    c.nbr = ctx->d_nbr.p;
    c.nao = ctx->d_nao.p;
    c.nabf = ctx->d_nabf.p;
    c.ncol = ctx->d_ncol.p;
    c.C = DevBlocks{ctx->K[0].data.p, ctx->K[0].d_offs.p, ctx->K[0].maxabs.p};
    c.V = DevBlocks{ctx->K[1].data.p, ctx->K[1].d_offs.p, ctx->K[1].maxabs.p};
    c.D = DevBlocks{ctx->K[2].data.p, ctx->K[2].d_offs.p, ctx->K[2].maxabs.p};
    c.dhash = DevHash{ctx->d_dhkeys.p, ctx->d_dhvals.p, ctx->dmask};
    c.shash = DevHash{ctx->d_shkeys.p, ctx->d_shvals.p, ctx->smask};
    c.masks = ctx->d_masks.p;
    c.wg_flags = ctx->d_wg.p;
    c.wf_flags = ctx->d_wf.p;
    c.scratch = ctx->d_scratch.p;
    c.y_off = ctx->d_waveoffs.p;
    c.p_off = ctx->d_waveoffs.p + nw;
    c.t3_off = c.q_off = c.y_off;
    c.acc = ctx->d_acc.p;
    c.macs = ctx->d_counters.p + 8;
    c.err = ctx->d_err.p;
    c.sym = 0;
    c.skip = 2u | 4u | 8u | 16u | 32u | 64u;  // Y only
    c.dcacc = dcacc.p;
    c.dv = dvout.p;
    int nl = 0;
    CK(launch_contract_fp64(c, st, nullptr, &nl));
    CK(launch_adjoint(c, st));
    CK(cudaStreamSynchronize(st));
    w0 = w1;
  }
  CK(launch_fx_to_double(dcacc.p, nC, dcout.p, st));
  unsigned herr = 0;
  CK(cudaMemcpyAsync(&herr, ctx->d_err.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  if (dC) CK(cudaMemcpyAsync(dC, dcout.p, sizeof(double) * nC, cudaMemcpyDeviceToHost, st));
  if (dV) CK(cudaMemcpyAsync(dV, dvout.p, sizeof(double) * nV, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (herr) return fail(ctx, HFX_E_CUDA, "adjoint kernels reported error " + std::to_string(herr));
  return HFX_OK;
}

hfx_status hfx_stats(const hfx_ctx *ctx, void *stats) {
  if (!ctx || !stats) return HFX_E_ARG;
  if (!ctx->results_valid) return HFX_E_STATE;
  std::memcpy(stats, &ctx->stats, sizeof(hfx_stats_v1));
  return HFX_OK;
}

}  // extern "C"

// ------------------------------------------------- steps next to the build

namespace {
bool finite_all(const double *x, int64_t n) {
  for (int64_t i = 0; i < n; ++i)
    if (!std::isfinite(x[i])) return false;
  return true;
}
}  // namespace

hfx_status hfx_density_from_eigvecs(hfx_ctx *ctx, int32_t nk, const double *kfrac,
                                    int32_t nbands, const double *coef, const double *occ,
                                    int64_t nkeys, const int32_t *keys, double *out,
                                    double *max_imag) {
  if (!ctx) return HFX_E_ARG;
  if (nk < 1 || nbands < 1 || nkeys < 0 || !kfrac || !coef || !occ || (nkeys > 0 && (!keys || !out)))
    return fail(ctx, HFX_E_ARG, "density: bad sizes or null pointers");
  const int natoms = ctx->natoms;
  std::vector<int32_t> aoff(natoms + 1, 0);
  for (int x = 0; x < natoms; ++x) aoff[x + 1] = aoff[x] + ctx->nao[x];
  const int64_t nb = aoff[natoms];
  std::vector<int64_t> doff(nkeys + 1, 0);
  for (int64_t e = 0; e < nkeys; ++e) {
    const int32_t *k = keys + 5 * e;
    if (k[0] < 0 || k[0] >= natoms || k[1] < 0 || k[1] >= natoms)
      return fail(ctx, HFX_E_ARG, "density: key atom out of range");
    for (int c = 2; c < 5; ++c)
      if (k[c] < -127 || k[c] > 127) return fail(ctx, HFX_E_ARG, "density: |n| > 127");
    doff[e + 1] = doff[e] + (int64_t)ctx->nao[k[0]] * ctx->nao[k[1]];
  }
  const int64_t ncoef = (int64_t)nk * nb * nbands * 2, nocc = (int64_t)nk * nbands;
  if (!finite_all(kfrac, 3 * (int64_t)nk) || !finite_all(coef, ncoef) || !finite_all(occ, nocc))
    return fail(ctx, HFX_E_ARG, "density: non-finite input");
  if (nkeys == 0) {
    if (max_imag) *max_imag = 0.0;
    return HFX_OK;
  }
  cudaStream_t st = ctx->stream;
  DevBuf<double> dk, dc, dq, dout;
  DevBuf<int32_t> dkeys, daoff, dnao;
  DevBuf<int64_t> ddoff;
  DevBuf<unsigned long long> dmax;
  CK(dk.reserve(3 * nk));
  CK(dc.reserve(ncoef));
  CK(dq.reserve(nocc));
  CK(dout.reserve(doff[nkeys]));
  CK(dkeys.reserve(5 * nkeys));
  CK(daoff.reserve(natoms + 1));
  CK(dnao.reserve(natoms));
  CK(ddoff.reserve(nkeys + 1));
  CK(dmax.reserve(1));
  CK(cudaMemcpyAsync(dk.p, kfrac, sizeof(double) * 3 * nk, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(dc.p, coef, sizeof(double) * ncoef, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(dq.p, occ, sizeof(double) * nocc, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(dkeys.p, keys, sizeof(int32_t) * 5 * nkeys, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(daoff.p, aoff.data(), sizeof(int32_t) * (natoms + 1), cudaMemcpyHostToDevice,
                     st));
  CK(cudaMemcpyAsync(dnao.p, ctx->nao.data(), sizeof(int32_t) * natoms, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ddoff.p, doff.data(), sizeof(int64_t) * (nkeys + 1), cudaMemcpyHostToDevice,
                     st));
  CK(cudaMemsetAsync(dmax.p, 0, sizeof(unsigned long long), st));
  CK(launch_density(nk, dk.p, (int)nb, nbands, dc.p, dq.p, nkeys, dkeys.p, daoff.p, dnao.p,
                    ddoff.p, dout.p, dmax.p, st));
  unsigned long long mbits = 0;
  CK(cudaMemcpyAsync(out, dout.p, sizeof(double) * doff[nkeys], cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&mbits, dmax.p, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (max_imag) std::memcpy(max_imag, &mbits, sizeof(double));
  return HFX_OK;
}

hfx_status hfx_sigma_k(hfx_ctx *ctx, int32_t nk, const double *kfrac, double *out) {
  if (!ctx) return HFX_E_ARG;
  if (nk < 1 || !kfrac || !out) return fail(ctx, HFX_E_ARG, "sigma_k: bad sizes or null pointers");
  if (!ctx->results_valid) return fail(ctx, HFX_E_STATE, "sigma_k: no build");
  if (!finite_all(kfrac, 3 * (int64_t)nk)) return fail(ctx, HFX_E_ARG, "sigma_k: non-finite k");
  const int natoms = ctx->natoms;
  if ((int64_t)nk * natoms * natoms > 2147483647ll)
    return fail(ctx, HFX_E_ARG, "sigma_k: too many k points for this cell");
  std::vector<int32_t> aoff(natoms + 1, 0);
  for (int x = 0; x < natoms; ++x) aoff[x + 1] = aoff[x] + ctx->nao[x];
  const int64_t nb = aoff[natoms], nkeys = (int64_t)ctx->sig_keys.size();
  const int64_t nout = (int64_t)nk * nb * nb * 2;
  cudaStream_t st = ctx->stream;
  DevBuf<double> dk, dout;
  DevBuf<int32_t> daoff, dnao;
  DevBuf<uint64_t> dkeys;
  DevBuf<int64_t> doffs;
  CK(dk.reserve(3 * nk));
  CK(dout.reserve(nout));
  CK(daoff.reserve(natoms + 1));
  CK(dnao.reserve(natoms));
  CK(dkeys.reserve(nkeys));
  CK(doffs.reserve(nkeys + 1));
  CK(cudaMemcpyAsync(dk.p, kfrac, sizeof(double) * 3 * nk, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(daoff.p, aoff.data(), sizeof(int32_t) * (natoms + 1), cudaMemcpyHostToDevice,
                     st));
  CK(cudaMemcpyAsync(dnao.p, ctx->nao.data(), sizeof(int32_t) * natoms, cudaMemcpyHostToDevice, st));
  if (nkeys > 0) {
    CK(cudaMemcpyAsync(dkeys.p, ctx->sig_keys.data(), sizeof(uint64_t) * nkeys,
                       cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(doffs.p, ctx->sig_offs.data(), sizeof(int64_t) * (nkeys + 1),
                       cudaMemcpyHostToDevice, st));
  }
  CK(launch_sigma_k(nk, dk.p, natoms, daoff.p, dnao.p, nkeys, dkeys.p, doffs.p, ctx->d_sigma.p,
                    nb, dout.p, st));
  CK(cudaMemcpyAsync(out, dout.p, sizeof(double) * nout, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return HFX_OK;
}
