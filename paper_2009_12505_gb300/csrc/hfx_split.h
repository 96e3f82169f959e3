// Arguments of the split-precision (HFX_OZAKI) kernels.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "hfx_internal.h"

// One tensor-core job: a 128 x 64 output tile of work item w over K tiles
// [k0, k0 + nk) of 32.
struct Job {
  int64_t w;
  int32_t mt, nt, k0, nk;
};

// One job of the D_FG / D_FB product: up to two column blocks (G index in
// N[B], piece 1 = D_FG or 2 = D_FB) of work item w, over the F entries
// [ent, ent + nent) of the union of their survivors.
struct ZcJob {
  int32_t w;
  int16_t g[2];
  int8_t piece[2];
  int8_t nblk;
  int8_t pad;
  int32_t nent;
  int32_t pad2;
  int64_t ent;
};

// One F of a job: its K offset and width in the A operand, and per column
// block the element offset of the D digit tile (-1: screened out, zeros).
struct ZcEnt {
  int32_t kofs, kb;
  int64_t dz[2];
};

// Per-build data: work items, screen output and the digit-sliced C and V.
struct SplitShared {
  int32_t natoms;
  int64_t nv;                      // V blocks (= work items)
  const int32_t *nao, *nabf, *ncol, *ktY, *kt4;
  const int64_t *nc_start;         // per atom: first neighbour entry (natoms + 1)
  const NbrEntry *nbr;
  const WorkItem *items;
  const double *Cd, *Vd;
  const int64_t *Co, *Vo;
  const uint32_t *masks;
  const uint8_t *wg;
  DevHash shash;
  unsigned long long *acc;
  unsigned *err;
  int32_t sym;
  // C of each atom transposed for Y: rows (b, G, g), K = beta
  __nv_bfloat16 *cy;
  const int64_t *cy_base, *cy_rowpre;
  int16_t *cy_e;
  // C of each atom as rows (F, f), K = (alpha, a)
  __nv_bfloat16 *c4;
  const int64_t *c4_base, *c4_rowpre;
  int16_t *c4_e;
  // V blocks: rows alpha, K = beta
  __nv_bfloat16 *vs;
  const int64_t *vs_base, *v_rowpre;
  int16_t *vs_e;
  // C of each atom as rows (alpha, a), K = F blocks of width kb(F) = 16 ceil(nao(F)/16)
  __nv_bfloat16 *cz;
  const int64_t *cz_base, *cz_rowpre;
  int16_t *cz_e;
  const int32_t *kofs;             // per neighbour entry: K offset of its F block
  const int32_t *ktotZ;            // per atom: total K of its F blocks
  const double *Dd;
  const int64_t *Do;
  DevHash dhash;
  // D blocks as transposed digit tiles for the D_FG / D_FB products
  __nv_bfloat16 *dz;
  const __nv_bfloat16 *dzero;      // zero tile (6 digits of 32 x 32)
  const int64_t *dz_off;           // per D block
  const int32_t *dij;              // per D block: (i, j)
  unsigned long long *de;          // per (atom, ao) column maximum (bit pattern)
  const int32_t *aoff;             // per atom: first (atom, ao) index
  int64_t h_nd;                    // D blocks
  int32_t nsm;                     // SMs of the device (persistent grids)
  int32_t pd_pairs;                // f32 pairs of k_pdig's dynamic shared memory
  const int16_t *colG;             // per (atom, column): local index of its neighbour entry
  const int64_t *coloff;           // per atom: first column in colG
  int64_t h_cy_rows, h_c4_rows, h_v_rows, h_cz_rows;  // host copies of the row totals
};

// Per-wave data.
struct SplitWave {
  int64_t w0;
  int32_t nw;
  double *scratch;
  const int64_t *y_off, *p_off;
  const int64_t *p_rowpre;         // padded P rows per item (0 without D_AB jobs), nw + 1
  __nv_bfloat16 *ps;
  const int64_t *ps_base;          // -1 without D_AB jobs
  int16_t *ps_e;
  const int64_t *y_candpre, *v4_candpre;
  const int64_t *y_perm;           // wave items in Y-job order (grouped by atom B), nw
  const int64_t *pg_candpre;       // per item: nG if it has D_AB jobs else 0, nw + 1
  int64_t h_pgcand;
  Job *jobs, *jobs4;
  int *njobs;                      // [0] Y jobs, [1] D_AB jobs, [2] Z jobs, [3] Z entries
  unsigned long long *tmacs;       // [0] Y, [1] D_AB, [2] Z: multiply-adds of the launched jobs
                                   // (per digit product, padding included); [3] Z: those that
                                   // are neither padding nor zero tiles
  int64_t h_ycand, h_v4cand, h_prows, h_v4jobs_max;
  // Y as (hi, lo) f32 pairs in 16-column blocks, [cb][al][b][16], for the
  // D_FG / D_FB product epilogues and P; written only when y2_on (the region exists)
  const int64_t *y2_off;
  int32_t y2_on;
  // FP64 Y: 1 = every item (read by the FP64 kernels); 2 = none
  int32_t y64_mode;
  // D_FG and D_FB products: job list and F entries
  ZcJob *zc_jobs;
  ZcEnt *zc_ents;
  int64_t h_zc_jobs;
  // 512 job keys (size class x cost): the plan's count pass histograms
  // them, the fill pass takes them as the start offsets of each key's range
  // (small class first, each class longest first)
  int *zc_keys;
  // per CTA of the D_FG / D_FB product launches (small class at [0, nsm),
  // the others at [nsm, 2 nsm)): busy time in ns
  long long *cta_ns;
};

cudaError_t split_slice_inputs(const SplitShared &S, int ks, cudaStream_t st);
cudaError_t split_slice_cz(const SplitShared &S, int ks, cudaStream_t st);
// D digit tiles (needs S.de zeroed); run whenever D changes.
cudaError_t split_dz_prepare(const SplitShared &S, int ks, cudaStream_t st);
// D_FG / D_FB job plan for one wave: fill == 0 counts jobs and entries into
// W.njobs[2], W.njobs[3] and histograms the jobs' cost keys into W.zc_keys
// (256 ints, zeroed by the caller); fill == 1 writes W.zc_jobs (longest first:
// W.zc_keys must then hold each key's start offset, keys in descending order)
// and W.zc_ents.
cudaError_t split_zc_plan(const SplitShared &S, const SplitWave &W, int fill, cudaStream_t st);
// Launch shape of the D_FG / D_FB products: widest F block (16 or 32),
// largest block output count, shared bytes of one staged Y block.
struct ZcPlanShape {
  int kbmax, nout_max, ybytes;
  int ybytes_small;  // staged Y bytes for jobs whose blocks have at most 16 AOs
};
// D_FG / D_FB products of one wave (after phase 0: needs the Y pairs).
cudaError_t split_zc_run(const SplitShared &S, const SplitWave &W, int ks, const ZcPlanShape &P,
                         int nsm, int nsmall, cudaStream_t st);
// Y products (job 0) or D_AB products (job 1) of the wave's job list,
// persistent over at most maxjobs jobs.
cudaError_t split_pgemm(const SplitShared &S, const SplitWave &W, int ks, int job,
                        int64_t maxjobs, cudaStream_t st);
// phase 0: Y jobs; phase 1: P slices and D_AB jobs
cudaError_t split_wave(const SplitShared &S, const SplitWave &W, int ks, int phase,
                       cudaStream_t st);
