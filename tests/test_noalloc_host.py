"""Host-side checks of the allocation-free correlation-energy entry point
(rteom_ecorr_noalloc), runnable without a GPU.

The entry point serves callers that cannot allocate device memory (their GPU
memory belongs to their own pool or framework allocator, or they run where a
cudaMalloc/cudaFree is not allowed).  Its scratch is a static device array
whose address is cached per CUDA context; these tests check that cache's key
on the CPU, and that sizes beyond the scratch are rejected before any CUDA
call is made.
"""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2301_04249_b300 import RTEOM_ERR_ARG, _lib

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_2301_04249_b300", "csrc")

CACHE_CHECK = r"""
#include <cstdio>
#include "scratch_cache.h"
int main() {
  rteom::ContextAddressCache c;
  int lookups = 0;
  char a, b;
  void* next = &a;
  auto lookup = [&](void** out) { ++lookups; *out = next; return 0; };
  void* p = nullptr;
  if (c.get(7, lookup, &p) || p != &a || lookups != 1) return 1;   // first use: looked up
  next = &b;
  if (c.get(7, lookup, &p) || p != &a || lookups != 1) return 2;   // same context: cached
  if (c.get(8, lookup, &p) || p != &b || lookups != 2) return 3;   // new context (reset): fresh
  auto failing = [&](void** out) { ++lookups; *out = nullptr; return 5; };
  if (c.get(9, failing, &p) != 5 || lookups != 3) return 4;         // error returned
  if (c.get(9, lookup, &p) || p != &b || lookups != 4) return 5;   // failure was not cached
  if (c.size() != 3) return 6;
  std::puts("ok");
  return 0;
}
"""


def test_scratch_address_cache_is_keyed_per_context(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    src = tmp_path / "cache_check.cc"
    src.write_text(CACHE_CHECK)
    exe = tmp_path / "cache_check"
    subprocess.check_call([cxx, "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)])
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.returncode, r.stdout)


def test_noalloc_rejects_sizes_beyond_scratch():
    lib = _lib.load()
    err = ctypes.create_string_buffer(256)
    rc = lib.rteom_ecorr_noalloc(65, 10, 0, None, None, None, None, None, err, 256)
    assert rc == RTEOM_ERR_ARG
    rc = lib.rteom_ecorr_noalloc(65, 10, 0, None, None, None, ctypes.c_void_p(16), None, err, 256)
    assert rc == RTEOM_ERR_ARG and b"4096" in err.value
    rc = lib.rteom_ecorr_noalloc(0, 10, 0, None, None, None, ctypes.c_void_p(16), None, err, 256)
    assert rc == RTEOM_ERR_ARG
