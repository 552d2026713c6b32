"""The CTA maps of the batched cooperative launches (host code, g++ only):
how a launch's CTAs are split among a batch's streams.  Streams of weight 0
get no CTA, every other stream at least one, all CTAs are used, each
stream's CTAs are contiguous and the split follows the weights to within one
CTA of the largest-remainder rounding."""
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1905_02082_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <vector>
#include "rf_cta_map.hpp"
int main() {
  int cases;
  if (std::scanf("%d", &cases) != 1) return 1;
  for (int c = 0; c < cases; ++c) {
    int n, total;
    if (std::scanf("%d %d", &n, &total) != 2) return 1;
    std::vector<double> w(n);
    for (auto& x : w) std::scanf("%lf", &x);
    std::vector<int> map(total + n + 1, -7);
    rf::fill_cta_map(w, total, map.data());
    for (int v : map) std::printf("%d ", v);
    std::printf("\n");
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    d = tmp_path_factory.mktemp("ctamap")
    src = d / "driver.cpp"
    src.write_text(DRIVER)
    exe = d / "driver"
    subprocess.run(["g++", "-O1", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    return str(exe)


def _run(driver, cases):
    text = f"{len(cases)}\n" + "".join(f"{len(w)} {t} " + " ".join(repr(float(x)) for x in w) + "\n"
                                       for w, t in cases)
    out = subprocess.run([driver], input=text, capture_output=True, text=True, check=True).stdout.splitlines()
    return [np.array(line.split(), dtype=np.int64) for line in out]


def test_maps_use_every_cta_and_follow_the_weights(driver):
    rng = np.random.default_rng(5)
    cases = []
    for _ in range(400):
        n = int(rng.integers(1, 40))
        w = rng.choice([0.0, 19200.0, 76800.0, 307200.0, 921600.0], size=n) * rng.integers(1, 3, size=n)
        if rng.random() < 0.5:
            w = w * (rng.random(n) < 0.7)  # idle and first-frame streams: weight 0
        active = int((w > 0).sum())
        total = int(rng.integers(max(active, 1), 300))
        cases.append((w, total))
    cases.append((np.zeros(5), 152))  # nothing tracked
    cases.append((np.full(152, 307200.0), 152))  # one CTA each
    for (w, total), m in zip(cases, _run(driver, cases)):
        n = len(w)
        cta, first = m[:total], m[total:]
        assert len(first) == n + 1 and first[0] == 0
        cnt = np.diff(first)
        active = w > 0
        assert np.all(cnt[~active] == 0) and np.all(cnt[active] >= 1)
        if active.any():
            assert first[n] == total  # every CTA has a stream
            spare = total - active.sum()
            share = spare * w[active] / w[active].sum()
            assert np.all(np.abs((cnt[active] - 1) - share) < 1.0 + 1e-9)
        else:
            assert first[n] == 0 and np.all(cta == -1)
        for i in range(n):  # contiguous groups in stream order
            assert np.all(cta[first[i]:first[i + 1]] == i)
        assert np.all(cta[first[n]:] == -1)
