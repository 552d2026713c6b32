// CTA maps of the batched cooperative launches (host code, no CUDA): how a
// launch's CTAs are split among the streams of a batch.
#pragma once

#include <algorithm>
#include <utility>
#include <vector>

namespace rf {

// CTA counts of one launch: streams of weight 0 get none, the others at least
// one and the rest in proportion to their weight (pixel count), largest
// remainders first (ties to the lower stream index).  The counts sum to
// `total` when at least one stream has weight > 0 and the number of such
// streams does not exceed `total` (the batch guarantees it).
inline std::vector<int> split_ctas(const std::vector<double>& weight, int total) {
  const int n = (int)weight.size();
  std::vector<int> cnt(n, 0);
  double wsum = 0.0;
  int active = 0;
  for (int i = 0; i < n; ++i)
    if (weight[i] > 0.0) {
      cnt[i] = 1;
      wsum += weight[i];
      ++active;
    }
  if (active == 0) return cnt;
  const int spare = total - active;
  std::vector<std::pair<double, int>> rem;
  int given = 0;
  for (int i = 0; i < n; ++i) {
    if (weight[i] <= 0.0) continue;
    const double share = spare * weight[i] / wsum;
    const int whole = (int)share;
    cnt[i] += whole;
    given += whole;
    rem.push_back({share - whole, i});
  }
  std::sort(rem.begin(), rem.end(), [](const std::pair<double, int>& x, const std::pair<double, int>& y) {
    return x.first != y.first ? x.first > y.first : x.second < y.second;
  });
  for (int k = 0; k < spare - given && k < (int)rem.size(); ++k) cnt[rem[k].second]++;
  return cnt;
}

// CTA map of one launch: cta_stream[0, total) holds the stream of each CTA
// (-1: none), then cta_stream[total + i] is the first CTA of stream i and
// cta_stream[total + n] the end of the last group (total + n + 1 ints).
inline void fill_cta_map(const std::vector<double>& w, int total, int* cta_stream) {
  const int n = (int)w.size();
  int* group_first = cta_stream + total;
  const std::vector<int> cnt = split_ctas(w, total);
  int c = 0;
  for (int i = 0; i < n; ++i) {
    group_first[i] = c;
    for (int k = 0; k < cnt[i]; ++k) cta_stream[c++] = i;
  }
  group_first[n] = c;
  for (; c < total; ++c) cta_stream[c] = -1;
}

}  // namespace rf
