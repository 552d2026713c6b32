"""The host FP16 conversions used by volume export/import in FP16 storage
(paper_1905_02082_gb300/csrc/rf_half.hpp) against numpy's IEEE binary16:
every one of the 65,536 half values to float, and floats to half (round to
nearest even) over normal, subnormal, tie, overflow and special cases."""
import os
import subprocess

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _tool(tmp_path):
    src = tmp_path / "half.cpp"
    src.write_text(r'''
#include <cstdio>
#include <cstdint>
#include "rf_half.hpp"
int main(int argc, char** argv) {
  FILE* in = std::fopen(argv[1], "rb");
  FILE* out = std::fopen(argv[2], "wb");
  for (uint32_t h = 0; h < 65536; ++h) {
    float f = rf::half_bits_to_float((uint16_t)h);
    std::fwrite(&f, 4, 1, out);
  }
  float f;
  while (std::fread(&f, 4, 1, in) == 1) {
    uint16_t h = rf::float_to_half_bits(f);
    std::fwrite(&h, 2, 1, out);
  }
  std::fclose(in);
  std::fclose(out);
  return 0;
}
''')
    exe = tmp_path / "half"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_1905_02082_gb300", "csrc"), str(src),
                    "-o", str(exe)], check=True)
    return exe


def test_host_half_conversions_match_ieee(tmp_path):
    exe = _tool(tmp_path)
    rng = np.random.default_rng(0)
    specials = np.array([0.0, -0.0, 1.0, -1.0, 65504.0, 65519.99, 65520.0, 70000.0, -70000.0, np.inf, -np.inf,
                         2.0 ** -24, 2.0 ** -25, 1.5 * 2.0 ** -25, 2.0 ** -26, 2.0 ** -14, 2.0 ** -14 - 2.0 ** -25,
                         0.1, 1.0 / 3.0, 1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -11], dtype=np.float32)
    halves = np.arange(65536, dtype=np.uint16).view(np.float16)
    fin = halves[np.isfinite(halves)].astype(np.float32)
    mids = ((fin[:-1].astype(np.float64) + fin[1:].astype(np.float64)) / 2).astype(np.float32)  # ties and near-ties
    xs = np.concatenate([specials, rng.uniform(-1.5, 1.5, 200000).astype(np.float32),
                         (rng.standard_normal(50000) * 1e-5).astype(np.float32), mids,
                         np.nextafter(mids, np.float32(np.inf)), np.nextafter(mids, np.float32(-np.inf))])
    inp, outp = tmp_path / "in.bin", tmp_path / "out.bin"
    xs.tofile(inp)
    subprocess.run([str(exe), str(inp), str(outp)], check=True)
    raw = np.fromfile(outp, dtype=np.uint8)
    to_float = raw[:65536 * 4].view(np.float32)
    to_half = raw[65536 * 4:].view(np.uint16)
    ref = np.arange(65536, dtype=np.uint16).view(np.float16).astype(np.float32)
    nan = np.isnan(ref)
    np.testing.assert_array_equal(to_float[~nan].view(np.uint32), ref[~nan].view(np.uint32))
    assert np.isnan(to_float[nan]).all()
    with np.errstate(over="ignore"):  # values beyond the half range round to infinity
        expect = xs.astype(np.float16).view(np.uint16)
    np.testing.assert_array_equal(to_half, expect)
