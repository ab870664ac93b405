// Grouped MU engine: many independent NMF problems advanced together, one
// pass launch per (row bucket, rank bucket) and one combine launch per
// iteration for all of them.  Used by the batched and serving forms.
#pragma once

#include <vector>

#include "ntt_internal.cuh"

namespace ntt {

// One problem of a grouped pass launch (device table entry).  For a tall
// unfolding (m > NTT_MAX_ROWS) one entry per row block: X and W point at the
// block's first row, m is the block's row count.
struct GProb {
  const void* X;     // m x n, row stride n, FP32 (or BF16 in the BF16 buckets)
  float* H;          // re x n, row stride n, updated in place
  const float* W;    // m x re
  const float* G;    // R x R (bucket R), zero outside the diagonal blocks
  float* part;       // S x E partials of [P ; Q]
  float* Y;          // tall phase A: re x n partial W^T X of this row block
  int64_t n;
  int m, re, blk;    // rows, ranks, rank block size
  int S;             // CTAs of this problem in its launch
  int cta0;          // first CTA of this problem in its launch
  int aligned;       // X and H rows start on 16 bytes: 16-byte copies
  int prow0, qrow0;  // partial rows of P (this block's first row) and of Q
  int E;             // partial stride (floats) = (qrow0 + R) x R
  int hasq;          // this entry also accumulates Q
};

// One problem of the grouped combine launch (device table entry).
struct GComb {
  const float* part;   // S x E partials, E = (MP + R) x R
  float* red;          // E reduced sums (FP32 from an FP64 combine)
  float* W;            // m x re, updated in place
  float* G;            // R x R, W^T W on the diagonal blocks
  unsigned* ticket;    // zero between launches
  double* obj;         // objective trace (obj[t] after iteration t) or NULL
  const double* xnorm2;   // ||X||^2 (FP64) when obj is set
  int S, MP, R, m, re, blk;
  int blk0, nblk;      // combine blocks of this problem
};

int group_mp_bucket(int m);     // 16, 32, ..., 512; -1 above NTT_MAX_ROWS
int group_r_bucket(int re);     // 8, 16, 32; -1 above NTT_MAX_RANK
int group_tile_cols(int MP, int R);
int group_ctas_per_sm(int MP, int R, bool xb);   // resident pass CTAs per SM
// mode 0: fused pass; 1: tall phase A (MP = 512 only); 2: tall phase B (MP = 512 only);
// xb: BF16 X rows (mode 0, MP <= 256, R = 16 or 32)
cudaError_t launch_gpass(int mode, int MP, int R, bool xb, const GProb* probs, const int* cta_prob, int ncta,
                         float eps, cudaStream_t st);
bool gpass_bf16_supported(int MP, int R);
int gpass_occupancy_bf16(int MP, int R);
cudaError_t launch_gpass_bf16(int MP, int R, const GProb* probs, const int* cta_prob, int ncta, float eps,
                              cudaStream_t st);
int gpass_occupancy_r8(int MP);
int gpass_occupancy_r16(int MP);
int gpass_occupancy_r32(int MP);
cudaError_t launch_gpass_r8(int mode, int MP, const GProb* probs, const int* cta_prob, int ncta, float eps,
                            cudaStream_t st);
cudaError_t launch_gpass_r16(int mode, int MP, const GProb* probs, const int* cta_prob, int ncta, float eps,
                             cudaStream_t st);
cudaError_t launch_gpass_r32(int mode, int MP, const GProb* probs, const int* cta_prob, int ncta, float eps,
                             cudaStream_t st);

// Tall unfolding: the H update of one problem from its row blocks' partial Y.
struct GTall {
  const float* Y;    // nb x re x n partial W^T X, block after block
  float* H;          // re x n
  const float* G;    // R x R
  int64_t n;
  int re, R, nb, blk0;
};

// Shapes, buckets and the scratch layout of one grouped run.
struct GroupPlan {
  struct Prob {
    int64_t n;
    int m, re, blk, R;
    int tall, nb, mb;                  // tall: nb row blocks of mb rows (the last one shorter)
    int xbf16;                         // X in BF16
    int qrow0, E, S, blk0, nblk;       // partial layout, CTAs per entry, combine blocks
    int tblk0, tnblk;                  // tall H-update blocks
    size_t g_off, red_off, part_off, y_off;   // plan scratch (bytes) when the plan owns it
  };
  struct Entry {
    int p, b, mode, bucket, cta0;
  };
  struct Bucket {
    int mode, MP, R, xb, ncta, cta_off;
  };
  std::vector<Prob> probs;
  std::vector<Entry> entries;
  std::vector<Bucket> buckets;
  int total_cta = 0, total_cblk = 0, ntall = 0, total_tblk = 0;
  bool own_scratch = true;
  size_t o_prob, o_comb, o_tall, o_cta, o_cblk, o_tblk;   // offsets inside the table block
  size_t off_tables, table_bytes;      // tables (one host-to-device copy)
  size_t off_tickets, bytes;           // scratch bytes in total (end offset)
};

struct GroupShape {
  int64_t n;
  int m, re, blk;
  int xbf16 = 0;     // X in BF16 (fused buckets up to 256 rows, ranks 9..32; 16-byte aligned rows)
};

// Per-problem device buffers.  G, red, part and Y are the problem's engine
// scratch when the plan does not own it (group_problem_scratch bytes, in that order).
struct GroupPtrs {
  const void* X;
  float* H;
  float* W;
  char* scratch;
  double* obj = nullptr;          // objective trace of this problem (Gram form, FP64) or NULL
  const double* xnorm2 = nullptr; // ||X||^2 when obj is set
};

// Plan a grouped run of `shapes` (re <= NTT_MAX_RANK, 1 <= blk <= re; m above
// NTT_MAX_ROWS runs as row blocks); `base` is the scratch offset the plan
// starts at.  fixed_split: every problem's CTA count (and so its reduction
// order) depends on its own shape only, not on the other problems.
// own_scratch: G, red, part and Y of every problem live in the plan's scratch;
// otherwise GroupPtrs::scratch supplies them.  split_div: problems sharing a
// launch get CTAs of 1/split_div of one wave's tile share each (1, 2, 4, 8).
ntt_status group_plan(const std::vector<GroupShape>& shapes, int sms, size_t base, bool fixed_split,
                      bool own_scratch, GroupPlan* out, int split_div = 4);

// Engine scratch of one problem under fixed_split (bytes, 256-byte multiple).
size_t group_problem_scratch(const GroupShape& shape, int sms);

// Write the device tables of a run (pointers into `scratch` and the problems'
// buffers) into host memory of plan.table_bytes.  Host only.
void group_fill_tables(const GroupPlan& plan, const GroupPtrs* ptrs, char* scratch, void* host_tables);

// The Gram launch and `iters` MU iterations of every problem, with the tables
// already on the device at `dev_tables` (plan.table_bytes).
ntt_status group_launch(const GroupPlan& plan, char* scratch, const char* dev_tables, int iters, float eps,
                        cudaStream_t st, int t0 = 0);

// `iters` MU iterations of every problem of the plan.  W and H hold the
// initial factors; `host_tables` is pinned host memory of plan.table_bytes
// that must stay untouched until the stream has passed this call's copy.
// (group_fill_tables, one host-to-device copy into the scratch, group_launch.)
ntt_status group_run(const GroupPlan& plan, const GroupPtrs* ptrs, char* scratch, void* host_tables,
                     int iters, float eps, cudaStream_t st, int t0 = 0);

}  // namespace ntt
