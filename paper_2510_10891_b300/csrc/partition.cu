// Partitions of a CSR matrix for the SpMV kernels (Partition, common.cuh):
// the host plan (row classes, staged runs, long-row chunks) and its device
// copy.  The plan decides which kernel path every row takes, so the SpMV
// kernels' traffic depends on this file and the kernel sources only.
#include <algorithm>
#include <cstring>
#include <vector>

#include "lp.h"

namespace scuc {

namespace {
template <typename T>
int palloc(T** p, size_t count) {
  void* q = nullptr;
  const int rc = dev_alloc_bytes(&q, (count ? count : 1) * sizeof(T));  // padded: aligned bulk copies
  *p = static_cast<T*>(q);
  return rc;
}
}  // namespace

// Host plan of a partition (see Partition): rows with more than long_min
// (<= kGroupRowMax) nonzeros are cut into chunks of kChunk entries when
// allow_long (otherwise rows above kGroupRowMax join the 32-thread list
// rows); other rows of kShortMax+1..kGroupRowMax nonzeros
// get a group of group_size_for(len, shape.ept) threads; runs of at least
// shape.min_run consecutive short rows are packed into staged blocks of <=
// kMaxRows rows / <= kNnzCap nonzeros (threads per row = largest power of
// two with gsz * rows <= kBlock), shorter runs go to 4-thread list rows.
// List classes run from 32 threads per row down to 4 (longest work first),
// then the staged blocks, then the long rows.
void plan_partition(const std::vector<int>& rp, int m, const PartShape& shape, bool allow_long, PartPlan* plan,
                    int long_min) {
  // Two passes over the rows: the first gives every row its class (a list
  // class 0..3, a long row, a short row of a staged run, or a short row in
  // no list), counting the list rows per class; the second writes the list
  // rows straight to their class's place, the staged runs and the chunks
  // in row order.  (Appending to four growing per-class lists and copying
  // them took three times as long for the 1.5M columns of a 13k-bus A^T.)
  constexpr unsigned char kLong = 254, kStaged = 255, kNone = 253;
  static thread_local std::vector<unsigned char> cls;  // per host thread, reused
  cls.assign(m, kNone);
  plan->clear();  // keeps the vectors' capacity (see build_partition)
  plan->chunk_ptr.assign(1, 0);
  int cnt[4] = {0, 0, 0, 0};
  auto list_class = [&](int len) {
    const int g = len > kGroupRowMax ? 32 : group_size_for(len, shape.ept);
    return g == 32 ? 0 : g == 16 ? 1 : g == 8 ? 2 : 3;
  };
  auto mark_run = [&](int a, int b) {  // short rows [a, b): staged, or 4-thread list rows if too few
    if (b <= a) return;
    const bool staged = b - a >= shape.min_run;
    if (!staged) cnt[3] += b - a;
    memset(cls.data() + a, staged ? kStaged : 3, b - a);
  };
  int run0 = 0;
  for (int r = 0; r < m; r++) {
    const int len = rp[r + 1] - rp[r];
    if (len <= kShortMax) continue;
    mark_run(run0, r);
    run0 = r + 1;
    if (len > long_min && allow_long) {
      cls[r] = kLong;
    } else {
      const int k = list_class(len);
      cls[r] = (unsigned char)k;
      cnt[k]++;
    }
  }
  mark_run(run0, m);
  int at[4];
  for (int k = 0, o = 0; k < 4; k++) {
    plan->cls_row[k] = at[k] = o;
    plan->cls_blk[k + 1] = plan->cls_blk[k] + (cnt[k] + (kBlock >> (5 - k)) - 1) / (kBlock >> (5 - k));
    o += cnt[k];
  }
  plan->cls_row[4] = at[3] + cnt[3];
  plan->listx.resize(plan->cls_row[4]);
  int4* L = plan->listx.data();
  for (int r = 0; r < m;) {
    const unsigned char c = cls[r];
    if (c < 4) {
      L[at[c]++] = make_int4(r, rp[r], rp[r + 1], 0);
      r++;
    } else if (c == kLong) {
      plan->long_rows.push_back(r);
      for (int e = rp[r]; e < rp[r + 1]; e += kChunk)
        plan->chunks.push_back(make_int2(e, std::min(rp[r + 1], e + kChunk)));
      plan->chunk_ptr.push_back((int)plan->chunks.size());
      r++;
    } else if (c == kStaged) {
      // a run of short rows: blocks of <= kMaxRows rows / <= kNnzCap nonzeros
      int b = r;
      while (b < m && cls[b] == kStaged) b++;
      while (r < b) {
        const int start = r;
        int nz = 0;
        while (r < b && r - start < kMaxRows && nz + (rp[r + 1] - rp[r]) <= kNnzCap) {
          nz += rp[r + 1] - rp[r];
          r++;
        }
        const int nr = r - start;
        int g = 1;
        while (g < 32 && g * 2 * nr <= kBlock) g *= 2;
        plan->desc.push_back(make_int4(start, rp[start], rp[r], (nr << 8) | g));
      }
    } else {
      r++;
    }
  }
}

// device copies of a planned partition (freed by free_partition)
int upload_partition(const PartPlan& plan, Partition* P) {
  *P = Partition{};
  for (int k = 0; k < 5; k++) {
    P->cls_blk[k] = plan.cls_blk[k];
    P->cls_row[k] = plan.cls_row[k];
  }
  P->nstaged = (int)plan.desc.size();
  P->nlong = (int)plan.long_rows.size();
  P->nchunk = (int)plan.chunks.size();
  P->nchunkblk = (P->nchunk + kBlock / 32 - 1) / (kBlock / 32);
  for (const int2& c : plan.chunks) P->nchunk_ent += c.y - c.x;
  P->nblk = plan.cls_blk[4] + P->nstaged + (P->nlong + kBlock - 1) / kBlock;
  SCUC_TRY(palloc(&P->listx, plan.listx.size()));
  SCUC_TRY(palloc(&P->desc, plan.desc.size()));
  SCUC_TRY(palloc(&P->chunks, plan.chunks.size()));
  SCUC_TRY(palloc(&P->long_rows, plan.long_rows.size()));
  SCUC_TRY(palloc(&P->chunk_ptr, plan.long_rows.size() + 1));
  SCUC_TRY(palloc(&P->cpart, plan.chunks.size()));
  SCUC_TRY(palloc(&P->crec, plan.chunks.size()));
  if (!plan.slot.empty()) SCUC_TRY(palloc(&P->slot, plan.slot.size()));
  auto up = [](void* dst, const void* src, size_t bytes) {
    return bytes ? cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice) : cudaSuccess;
  };
  SCUC_CUDA(up(P->listx, plan.listx.data(), plan.listx.size() * sizeof(int4)));
  SCUC_CUDA(up(P->desc, plan.desc.data(), plan.desc.size() * sizeof(int4)));
  SCUC_CUDA(up(P->chunks, plan.chunks.data(), plan.chunks.size() * sizeof(int2)));
  SCUC_CUDA(up(P->long_rows, plan.long_rows.data(), plan.long_rows.size() * sizeof(int)));
  SCUC_CUDA(up(P->chunk_ptr, plan.chunk_ptr.data(), plan.chunk_ptr.size() * sizeof(int)));
  if (P->slot) SCUC_CUDA(up(P->slot, plan.slot.data(), plan.slot.size() * sizeof(int)));
  return SCUC_OK;
}

void free_partition(Partition* P) {
  for (void* q : {(void*)P->listx, (void*)P->desc, (void*)P->chunks, (void*)P->long_rows, (void*)P->chunk_ptr,
                  (void*)P->cpart, (void*)P->slot, (void*)P->cst, (void*)P->crec})
    if (q) dev_free(q);
  *P = Partition{};
}

// Sliced ELL structure (Sell, common.cuh): the rows of at most max_len
// nonzeros (longer rows are left out: no lane computes them), sorted by
// length (longest first, ties by index) within windows of kSellWindow rows
// and cut into slices of 32; slices ordered longest first (the longest
// start first, so the launch ends evenly).
int build_sell(const std::vector<int>& rp, int m, int max_len, Sell* S, std::vector<void*>* allocs) {
  *S = Sell{};
  struct Slice {
    int len;
    int first;  // index into order
    int end;    // end of its window's rows in order
  };
  std::vector<int> order(m > 0 ? m : 1);
  std::vector<Slice> slices;
  // rows of each window ordered by length, longest first, ties by index: a
  // stable counting sort over the lengths 0..max_len (a comparison sort of
  // the 1.5M columns of a 13k-bus A^T took 30 ms on the host)
  std::vector<int> cnt(max_len + 2);
  int kept = 0;
  for (int w0 = 0; w0 < m; w0 += kSellWindow) {
    const int w1 = std::min(m, w0 + kSellWindow);
    const int k0 = kept;
    std::fill(cnt.begin(), cnt.end(), 0);
    for (int r = w0; r < w1; r++) {
      const int len = rp[r + 1] - rp[r];
      if (len <= max_len) cnt[len]++;
    }
    int at = k0;
    for (int len = max_len; len >= 0; len--) {  // cnt[len] becomes the first place of length len
      const int c = cnt[len];
      cnt[len] = at;
      at += c;
    }
    for (int r = w0; r < w1; r++) {
      const int len = rp[r + 1] - rp[r];
      if (len <= max_len) order[cnt[len]++] = r;
    }
    kept = at;
    for (int q = k0; q < kept; q += 32) slices.push_back(Slice{rp[order[q] + 1] - rp[order[q]], q, kept});
  }
  std::stable_sort(slices.begin(), slices.end(), [](const Slice& a, const Slice& b) { return a.len > b.len; });
  const int ns = (int)slices.size();
  std::vector<int> sptr(ns + 1, 0), pptr(ns + 1, 0), rows((size_t)ns * 32, -1);
  for (int k = 0; k < ns; k++) {
    const Slice& sl = slices[k];
    for (int l = 0; l < 32 && sl.first + l < sl.end; l++) rows[(size_t)k * 32 + l] = order[sl.first + l];
    if ((int64_t)sptr[k] + sl.len > (int64_t)INT32_MAX / 32) {
      set_error("sliced ELL copy of %d rows exceeds 2^31 entries", m);
      return SCUC_E_INVALID;
    }
    sptr[k + 1] = sptr[k] + sl.len;
    pptr[k + 1] = pptr[k] + (sl.len + 1) / 2;
  }
  S->nslice = ns;
  S->nent = (int64_t)sptr[ns] * 32;
  SCUC_TRY(palloc(&S->sptr, sptr.size()));
  allocs->push_back(S->sptr);
  SCUC_TRY(palloc(&S->rows, rows.size()));
  allocs->push_back(S->rows);
  S->npair = pptr[ns];
  SCUC_TRY(palloc(&S->pptr, pptr.size()));
  allocs->push_back(S->pptr);
  SCUC_TRY(palloc(&S->col, (size_t)S->nent));
  allocs->push_back(S->col);
  SCUC_TRY(palloc(&S->v64, (size_t)S->nent));
  allocs->push_back(S->v64);
  SCUC_CUDA(cudaMemcpy(S->sptr, sptr.data(), sptr.size() * sizeof(int), cudaMemcpyHostToDevice));
  SCUC_CUDA(cudaMemcpy(S->rows, rows.data(), rows.size() * sizeof(int), cudaMemcpyHostToDevice));
  SCUC_CUDA(cudaMemcpy(S->pptr, pptr.data(), pptr.size() * sizeof(int), cudaMemcpyHostToDevice));
  return SCUC_OK;
}

int build_partition(const std::vector<int>& rp, int m, Partition* P, int long_min) {
  // per host thread and reused: a fixing round plans a new LP of a million
  // rows, whose freshly allocated plan arrays (16 MB) cost more in page
  // faults than filling them
  static thread_local PartPlan plan;
  plan_partition(rp, m, PartShape{}, true, &plan, long_min);
  return upload_partition(plan, P);
}

}  // namespace scuc
