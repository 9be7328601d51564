"""The leaf kernel's register sorting networks, checked on the host.

The kernel sorts its seed lists and parked values with Batcher's odd-even merge
sort, built at compile time as a comparator table (`OddEvenNet<N>` in the leaf
kernel's header).  The table is host-usable C++, so a small host program built
with nvcc applies it to every 0/1 input (0-1 principle: a comparator network
that sorts all 0/1 sequences sorts every sequence) for the sizes the kernel uses
(8 and 12 parking slots, 8/16/32/64-value lists), plus random float inputs
against std::sort.  No GPU is needed.
"""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2512_10386_gb300", "csrc")

PROGRAM = r"""
#include "gd_leaf_kernel.cuh"
#include <algorithm>
#include <cstdio>
#include <random>

template <int N>
static bool sorts(const float *in) {
  constexpr gd::OddEvenNet<N> net{};
  float v[N];
  for (int i = 0; i < N; ++i) v[i] = in[i];
  for (int c = 0; c < gd::OddEvenNet<N>::C; ++c) {
    const float x = v[net.a[c]], y = v[net.b[c]];
    v[net.a[c]] = x < y ? x : y;
    v[net.b[c]] = x < y ? y : x;
  }
  for (int i = 1; i < N; ++i)
    if (v[i - 1] > v[i]) return false;
  return true;
}

template <int N>
static int check(unsigned long long zero_one_limit) {
  float in[N];
  // every 0/1 input up to 2^20 of them, else a seeded sample
  const bool all = N <= 20;
  std::mt19937_64 rng(7);
  const unsigned long long cases = all ? (1ull << N) : zero_one_limit;
  for (unsigned long long m = 0; m < cases; ++m) {
    const unsigned long long bits = all ? m : rng();
    for (int i = 0; i < N; ++i) in[i] = (float)((bits >> (i % 64)) & 1ull);
    if (!sorts<N>(in)) { std::printf("N=%d 0/1 case %llu unsorted\n", N, m); return 1; }
  }
  std::uniform_real_distribution<float> u(-1.f, 1.f);
  for (int t = 0; t < 20000; ++t) {
    for (int i = 0; i < N; ++i) in[i] = (t & 1) ? u(rng) : (float)(rng() % 5);  // also many equal keys
    if (!sorts<N>(in)) { std::printf("N=%d random case %d unsorted\n", N, t); return 1; }
  }
  std::printf("N=%d comparators=%d ok\n", N, gd::OddEvenNet<N>::C);
  return 0;
}

int main() {
  int bad = 0;
  bad |= check<8>(0);
  bad |= check<12>(0);
  bad |= check<16>(0);
  bad |= check<32>(200000);
  bad |= check<64>(200000);
  return bad;
}
"""


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


def test_odd_even_networks_sort(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    src = tmp_path / "nets.cu"
    exe = tmp_path / "nets"
    src.write_text(PROGRAM)
    r = subprocess.run([nvcc, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "include"), "-I", CSRC, str(src),
                        "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    counts = dict(line.split()[0:2] for line in r.stdout.splitlines())
    # Batcher's odd-even merge sort sizes (fewer comparators than the bitonic 24 / 240)
    assert counts["N=8"] == "comparators=19" and counts["N=32"] == "comparators=191"
