// ce_plan.h -- the host-side launch models behind the automatic launch
// parameters: the z-sweep kernel's z-chunk count and the row kernel's item
// length on a single lattice.  Plain C++ (no CUDA), so the CPU tests compile
// it too.
#pragma once

#include <algorithm>
#include <cstdint>
#include <queue>
#include <utility>
#include <vector>

namespace ce {
namespace plan {

constexpr int kRowWarps = 8;   // warps per CTA of the row (batched) kernel

// Lanes per 3D row segment, as log2: the segment width (32, 16 or 8 lanes x VX
// sites) that pads a row of N sites least, the widest on a tie.  Depends on N
// only, so a lattice's items do not depend on the rest of the batch.
inline int seg_log2_for(int N, int VX) {
  int best = 5;
  int64_t best_pad = INT64_MAX;
  for (int sl = 5; sl >= 3; --sl) {
    const int64_t W = (int64_t)VX << sl;
    const int64_t pad = (N + W - 1) / W * W;
    if (pad < best_pad) {
      best_pad = pad;
      best = sl;
    }
  }
  return best;
}

// Items build_tables cuts a lattice into (same loops, counted).
inline int64_t item_count(int dims, int64_t N, int VX, int sweep_len) {
  const int64_t L = std::max<int64_t>(1, std::min<int64_t>(sweep_len, N));
  const int64_t span = kRowWarps * 32 * VX;
  if (dims == 3) {
    const int sl = seg_log2_for((int)N, VX);
    const int64_t W = (int64_t)VX << sl, rows = (int64_t)kRowWarps << (5 - sl);
    return ((N + W - 1) / W) * ((N + rows - 1) / rows) * ((N + L - 1) / L);
  }
  if (dims == 2) return ((N + span - 1) / span) * ((N + L - 1) / L);
  return (N + span - 1) / span;
}

// Predicted duration, in plane-times, of one launch on a lattice alone cut into
// items of L planes along the sweep axis (plus two halo planes and a start-up
// cost of about two planes each), taken from the queue in build order by
// `slots` resident CTAs.  The active CTAs share HBM equally and one CTA streams
// at most 1.25x its share under full load: a processor-sharing model whose two
// constants were chosen on timings of single 2D and 3D lattices (a lattice of
// few columns needs short items to keep the CTAs busy, a large one long items
// to amortise the halo planes, and a fraction of a wave costs a whole item).
inline double rows_predicted_time(int dims, int64_t N, int VX, int L, int slots) {
  const int64_t Lc = std::max<int64_t>(1, std::min<int64_t>(L, N));
  const int64_t nz = (N + Lc - 1) / Lc, last = N - (nz - 1) * Lc;
  const int64_t cols = item_count(dims, N, VX, (int)N);   // items of one full-length chunk
  const int64_t n = cols * nz;
  // 3D items run z-chunk by z-chunk (the short last chunk at the end), 2D items column by column
  auto planes = [&](int64_t k) -> double {
    const bool tail = dims == 3 ? k >= cols * (nz - 1) : (k % nz) == nz - 1;
    return (double)((tail ? last : Lc) + 2 + 2);
  };
  constexpr double kSoloSpeedup = 1.25;
  std::vector<double> rem;
  rem.reserve(slots);
  int64_t next = 0;
  while (next < n && (int)rem.size() < slots) rem.push_back(planes(next++));
  double t = 0.0;
  while (!rem.empty()) {
    const double rate = std::min(kSoloSpeedup, (double)slots / (double)rem.size());
    const double m = *std::min_element(rem.begin(), rem.end());
    t += m / rate;
    size_t keep = 0;
    for (size_t i = 0; i < rem.size(); ++i)
      if (rem[i] - m > 1e-9) rem[keep++] = rem[i] - m;
    size_t freed = rem.size() - keep;
    rem.resize(keep);
    for (; freed > 0 && next < n; --freed) rem.push_back(planes(next++));
  }
  return t;
}

// Item length of a lattice alone: the candidate with the least predicted time
// (ties to the longer item).  1D lattices are one row; their items do not depend on it.
inline int rows_item_length(int dims, int64_t N, int VX, int slots) {
  static const int kCand[] = {128, 96, 64, 48, 32, 24, 16, 12, 8, 4};
  if (dims == 1) return 128;
  int best = 128;
  double best_t = -1.0;
  for (int L : kCand) {
    if (L > N && L != 128) continue;
    const double t = rows_predicted_time(dims, N, VX, L, slots);
    if (best_t < 0.0 || t < best_t * (1.0 - 1e-3)) {
      best_t = t;
      best = L;
    }
  }
  return best;
}


// Predicted duration (in plane-times of a CTA sharing its SM) of a launch of
// cols x gz CTAs, each sweeping its chunk of N / gz planes plus 2 halo planes
// and a start-up of about 4 planes.  Blocks are handed out in grid order to the
// SM slots that free up; a CTA runs 1.32x faster while it is alone on its SM
// (ncu: 2.2k against 2.9k cycles per plane at 256^3), and an SM never streams
// faster than per_sm CTAs sharing it.  The lone-CTA speed-up is what makes a
// partial wave cheaper than a whole one: at 256^3 the model prefers 4 chunks
// (0.84 of a wave; measured 93.3 us) to 14 (101.6 us), which a count of whole
// waves would pick.  Event-driven: one heap entry per SM.
inline double grid_time(int64_t N, int64_t cols, int gz, int per_sm, int sms) {
  constexpr double kStart = 4.0, kSolo = 1.32;
  const double cap = (double)per_sm;
  auto rate = [&](size_t n) { return std::min(kSolo, cap / (double)n); };
  const int64_t nblk = cols * gz;
  auto work = [&](int64_t b) {
    const int64_t zc = b / cols;
    return (double)((zc + 1) * N / gz - zc * N / gz + 2) + kStart;
  };
  std::vector<std::vector<double>> rem(sms);
  std::vector<double> last(sms, 0.0);
  int64_t next = 0;
  for (int r = 0; r < per_sm; ++r)
    for (int s = 0; s < sms && next < nblk; ++s) rem[s].push_back(work(next++));
  using Ev = std::pair<double, int>;
  std::priority_queue<Ev, std::vector<Ev>, std::greater<Ev>> heap;
  for (int s = 0; s < sms; ++s)
    if (!rem[s].empty()) heap.push({*std::min_element(rem[s].begin(), rem[s].end()) / rate(rem[s].size()), s});
  double end = 0.0;
  while (!heap.empty()) {
    const auto [t, s] = heap.top();
    heap.pop();
    const double done = (t - last[s]) * rate(rem[s].size());
    size_t keep = 0, freed = 0;
    for (double w : rem[s]) {
      if (w - done > 1e-9) rem[s][keep++] = w - done;
      else ++freed;
    }
    rem[s].resize(keep);
    for (; freed > 0 && next < nblk; --freed) rem[s].push_back(work(next++));
    last[s] = t;
    end = std::max(end, t);
    if (!rem[s].empty()) heap.push({t + *std::min_element(rem[s].begin(), rem[s].end()) / rate(rem[s].size()), s});
  }
  return end;
}

// The automatic z-chunk count of the z-sweep kernel: among chunks of at most
// 64 planes, the count with the least predicted launch time (grid_time).
// Longer chunks measured slower on large lattices than the model says (640^3:
// 3 chunks 1363 us, 12 chunks 1279 us); with the cap the pick was the measured
// best, or within 1-5% of it, on every FP32 lattice timed (128^3 to 1024^3, 8-
// and 16-row tiles).
inline int auto_zchunks(int64_t N, int64_t cols, int per_sm, int sms) {
  constexpr int kMaxChunk = 64;
  const int gz_min = (int)std::max<int64_t>(1, (N + kMaxChunk - 1) / kMaxChunk);
  double best = 1e300;
  int best_gz = (int)std::min<int64_t>(gz_min, N / 2);
  for (int gz = gz_min; gz <= N / 4 && gz <= 128; ++gz) {
    if (gz > gz_min && cols * gz > 32LL * per_sm * sms) break;   // 32 waves: no tail left to win
    const double t = grid_time(N, cols, gz, per_sm, sms);
    if (t < best * (1.0 - 1e-6)) {
      best = t;
      best_gz = gz;
    }
  }
  return best_gz;
}

// Chunk length along the sweep axis for the kernels whose blocks each sweep one
// chunk of an N-long axis (the column kernel's z-chunks, the line-sweep
// kernel's row chunks): the length with the least predicted time, where the
// launch's blocks (`blocks_per_chunk` per chunk) run in waves of `slots`
// resident blocks and each wave costs its chunk plus `overhead` planes (the 2
// halo planes and the start-up), a partial wave costing a whole one.  Chunks of
// at least `min_len` planes (fewer chunks on a tie).
inline int wave_chunk_length(int64_t N, int64_t blocks_per_chunk, int64_t slots, int64_t min_len,
                             double overhead) {
  double best = 1e300;
  int64_t best_len = N;
  for (int64_t gz = 1; gz <= std::max<int64_t>(1, N / min_len); ++gz) {
    const int64_t len = (N + gz - 1) / gz, chunks = (N + len - 1) / len;
    const int64_t waves = (blocks_per_chunk * chunks + slots - 1) / slots;
    const double t = (double)waves * ((double)len + overhead);
    if (t < best * (1.0 - 1e-9)) {
      best = t;
      best_len = len;
    }
  }
  return (int)best_len;
}

}  // namespace plan
}  // namespace ce
