"""Host policy of the serving form (csrc/serve_policy.h), compiled with the
host C++ compiler and checked against a brute-force model: the arena never
hands out overlapping blocks, keeps exact byte counts, merges free neighbours;
admission is FIFO by arrival, gated by free slots and the budget."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2008_01340_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>
#include "serve_policy.h"
using namespace ntt::serve;
#define CHECK(c) do { if (!(c)) { std::printf("FAIL line %d: %s\n", __LINE__, #c); return 1; } } while (0)

int main() {
  // ---- deterministic arena cases
  Arena a(1 << 20);
  CHECK(a.capacity() == (1u << 20));
  CHECK(a.alloc(0) == -1);
  CHECK(a.alloc((1 << 20) + 1) == -1);
  int64_t b0 = a.alloc(1000), b1 = a.alloc(300), b2 = a.alloc(256);
  CHECK(b0 == 0 && b1 == 1024 && b2 == 1024 + 512);       // 256-byte granules, first fit
  CHECK(a.in_use() == 1024 + 512 + 256);
  CHECK(a.release(b1));
  CHECK(!a.release(b1));                                   // not live any more
  CHECK(!a.release(12345));
  CHECK(a.alloc(200) == 1024);                             // reuses the hole
  CHECK(a.release(1024) && a.release(b0) && a.release(b2));
  CHECK(a.in_use() == 0 && a.free_ranges() == 1 && a.largest_free() == (1u << 20));
  CHECK(a.peak() == 1024 + 512 + 256);

  // ---- random stress against a byte map
  std::mt19937_64 rng(7);
  const size_t cap = 1 << 16;
  Arena r(cap);
  std::vector<int> owner(cap, -1);
  std::vector<std::pair<int64_t, size_t>> live;
  size_t used = 0;
  for (int step = 0; step < 20000; ++step) {
    if (live.empty() || rng() % 3) {
      const size_t want = 1 + rng() % 3000;
      const int64_t off = r.alloc(want);
      const size_t len = (want + 255) / 256 * 256;
      if (off < 0) {
        // first fit failed: no free run of len bytes may exist
        size_t run = 0, best = 0;
        for (size_t i = 0; i < cap; ++i) { run = owner[i] < 0 ? run + 1 : 0; best = run > best ? run : best; }
        CHECK(best < len);
        continue;
      }
      CHECK(off % 256 == 0 && (size_t)off + len <= cap);
      for (size_t i = 0; i < len; ++i) { CHECK(owner[off + i] < 0); owner[off + i] = step; }
      live.push_back({off, len});
      used += len;
    } else {
      const size_t k = rng() % live.size();
      CHECK(r.release(live[k].first));
      for (size_t i = 0; i < live[k].second; ++i) owner[live[k].first + i] = -1;
      used -= live[k].second;
      live.erase(live.begin() + k);
    }
    CHECK(r.in_use() == used);
  }
  for (auto& b : live) CHECK(r.release(b.first));
  CHECK(r.in_use() == 0 && r.free_ranges() == 1);

  // ---- admission: FIFO, slots, budget, head-of-line, too-large heads rejected
  Arena q(10000 * 256);
  AdmissionQueue Q;
  Q.push(1, 4000 * 256);
  Q.push(2, 5000 * 256);
  Q.push(3, 2000 * 256);     // fits only after 1 or 2 leave
  Q.push(4, 20000 * 256);    // larger than the arena: rejected when it reaches the head
  Q.push(5, 100 * 256);
  std::vector<int64_t> adm, rej;
  std::vector<int64_t> offs(8, -1);
  auto A = [&](int64_t id, int64_t off) { adm.push_back(id); offs[id] = off; };
  auto J = [&](int64_t id) { rej.push_back(id); };
  CHECK(Q.admit(q, 8, A, J) == 2);
  CHECK(adm.size() == 2 && adm[0] == 1 && adm[1] == 2 && Q.size() == 3);   // 5 waits behind 3
  CHECK(Q.admit(q, 8, A, J) == 0);
  CHECK(q.release(offs[1]));
  CHECK(Q.admit(q, 1, A, J) == 1 && adm.back() == 3);                      // one slot only
  CHECK(Q.admit(q, 4, A, J) == 1 && adm.back() == 5 && rej.size() == 1 && rej[0] == 4);
  CHECK(Q.empty());
  std::printf("OK\n");
  return 0;
}
"""


def test_serve_policy_host_logic(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "driver.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "driver"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip().endswith("OK"), out.stdout + out.stderr
