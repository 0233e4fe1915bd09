"""The per-context memo of the allocation-free entry point's scratch
address (csrc/sht_ctx_cache.h), compiled with the host C++ compiler and run
without a GPU: addresses are kept per context, a fresh lookup replaces a
stale one (a context re-created after a device reset may load the module
elsewhere), a call under stream capture uses the remembered address and
fails cleanly when its context has none, and a failed lookup is reported."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_1711_11296_gb300", "csrc")

SRC = r'''
#include <cstdio>
#include "sht_ctx_cache.h"
using namespace sht;
#define CHECK(c) do { if (!(c)) { std::printf("FAIL line %d\n", __LINE__); return 1; } } while (0)
int main() {
    ContextAddressCache<3> cache;
    char c1, c2, c3, c4;                  // stand-ins for four contexts
    char a1, a2, a3, a4, a1b;             // stand-ins for device addresses
    void* out = nullptr;
    int lookups = 0;
    auto give = [&](void* a) { return [&, a](void** p) { ++lookups; *p = a; return 0; }; };
    // capture before any uncaptured call in the context: refused, no lookup
    CHECK(scratch_for_context(cache, &c1, true, give(&a1), &out) == kScratchNeedsSetup);
    CHECK(lookups == 0);
    // uncaptured calls look up and remember per context
    CHECK(scratch_for_context(cache, &c1, false, give(&a1), &out) == kScratchOk && out == &a1);
    CHECK(scratch_for_context(cache, &c2, false, give(&a2), &out) == kScratchOk && out == &a2);
    CHECK(lookups == 2);
    // captured calls use the remembered address of their own context
    CHECK(scratch_for_context(cache, &c1, true, give(&a4), &out) == kScratchOk && out == &a1);
    CHECK(scratch_for_context(cache, &c2, true, give(&a4), &out) == kScratchOk && out == &a2);
    CHECK(lookups == 2);
    // every uncaptured call looks up again: a stale address is replaced
    CHECK(scratch_for_context(cache, &c1, false, give(&a1b), &out) == kScratchOk && out == &a1b);
    CHECK(scratch_for_context(cache, &c1, true, give(&a4), &out) == kScratchOk && out == &a1b);
    // a failed lookup is reported and remembers nothing
    auto fail = [&](void** p) { *p = nullptr; return 1; };
    CHECK(scratch_for_context(cache, &c3, false, fail, &out) == kScratchLookupFailed);
    CHECK(cache.get(&c3) == nullptr);
    // full: the oldest entry makes room
    CHECK(scratch_for_context(cache, &c3, false, give(&a3), &out) == kScratchOk);
    CHECK(scratch_for_context(cache, &c4, false, give(&a4), &out) == kScratchOk);
    CHECK(cache.get(&c4) == &a4 && cache.get(&c1) == nullptr);
    CHECK(cache.get(&c2) == &a2 && cache.get(&c3) == &a3);
    std::printf("ok\n");
    return 0;
}
'''


def test_context_address_cache(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "cache_check.cpp"
    src.write_text(SRC)
    exe = tmp_path / "cache_check"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", HDR, str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
