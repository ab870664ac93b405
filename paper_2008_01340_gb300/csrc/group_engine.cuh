// Grouped MU engine: many independent NMF problems advanced together, one
// pass launch per (row bucket, rank bucket) and one combine launch per
// iteration for all of them.  Used by the batched and serving forms.
#pragma once

#include <vector>

#include "ntt_internal.cuh"

namespace ntt {

// One problem of a grouped pass launch (device table entry).
struct GProb {
  const float* X;    // m x n, row stride n
  float* H;          // re x n, row stride n, updated in place
  const float* W;    // m x re
  const float* G;    // R x R (bucket R), zero outside the diagonal blocks
  float* part;       // S x (MP + R) x R partials of [P ; Q]
  int64_t n;
  int m, re, blk;    // rows, ranks, rank block size
  int S;             // CTAs of this problem in its launch
  int cta0;          // first CTA of this problem in its launch
  int aligned;       // X and H rows start on 16 bytes: 16-byte copies
  int pad[2];
};

// One problem of the grouped combine launch (device table entry).
struct GComb {
  const float* part;   // S x E partials, E = (MP + R) x R
  float* red;          // E reduced sums (FP32 from an FP64 combine)
  float* W;            // m x re, updated in place
  float* G;            // R x R, W^T W on the diagonal blocks
  unsigned* ticket;    // zero between launches
  int S, MP, R, m, re, blk;
  int blk0, nblk;      // combine blocks of this problem
};

int group_mp_bucket(int m);     // 16, 32, ..., 512; -1 above NTT_MAX_ROWS
int group_r_bucket(int re);     // 8, 16, 32; -1 above NTT_MAX_RANK
int group_tile_cols(int MP, int R);
cudaError_t launch_gpass(int MP, int R, const GProb* probs, const int* cta_prob, int ncta, float eps,
                         cudaStream_t st);
cudaError_t launch_gpass_r8(int MP, const GProb* probs, const int* cta_prob, int ncta, float eps,
                            cudaStream_t st);
cudaError_t launch_gpass_r16(int MP, const GProb* probs, const int* cta_prob, int ncta, float eps,
                             cudaStream_t st);
cudaError_t launch_gpass_r32(int MP, const GProb* probs, const int* cta_prob, int ncta, float eps,
                             cudaStream_t st);

// Shapes, buckets and the scratch layout of one grouped run.
struct GroupPlan {
  struct Prob {
    int64_t n;
    int m, re, blk;
    int MP, R, S, cta0, bucket, blk0, nblk;
    size_t part_off, red_off, g_off;   // bytes into the scratch
    int aligned_hint;                  // caller promises 16-byte rows (checked again at run time)
  };
  struct Bucket {
    int MP, R, ncta, cta_off;
  };
  std::vector<Prob> probs;
  std::vector<Bucket> buckets;
  int total_cta = 0, total_cblk = 0;
  size_t off_tables, table_bytes;      // GProb[], GComb[], CTA map, combine-block map
  size_t off_tickets, bytes;           // scratch bytes in total
};

struct GroupShape {
  int64_t n;
  int m, re, blk;
};

struct GroupPtrs {
  const float* X;
  float* H;
  float* W;
};

// Plan a grouped run of `shapes` (m <= NTT_MAX_ROWS, re <= NTT_MAX_RANK,
// 1 <= blk <= re); `base` is the scratch offset the plan starts at.
ntt_status group_plan(const std::vector<GroupShape>& shapes, int sms, size_t base, GroupPlan* out);

// `iters` MU iterations of every problem of the plan.  W and H hold the
// initial factors; `host_tables` is pinned host memory of plan.table_bytes
// that must stay untouched until the stream has passed this call's copy.
ntt_status group_run(const GroupPlan& plan, const GroupPtrs* ptrs, char* scratch, void* host_tables,
                     int iters, float eps, cudaStream_t st);

}  // namespace ntt
