"""Build libkb.so in-tree with nvcc for sm_103a (one -gencode, units compiled in parallel)."""

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libkb.so")
# the bounds-checked variant (-DKB_CHECKED), built on request into its own folder
OUT_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(OUT_CHECKED, "libkb.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _stale(lib):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(HERE, "..", "include", "kb.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False, checked=False):
    out, lib = (OUT_CHECKED, LIB_CHECKED) if checked else (OUT, LIB)
    flags = FLAGS + (["-DKB_CHECKED"] if checked else [])
    os.makedirs(out, exist_ok=True)
    srcs = sources()
    objs = [os.path.join(out, os.path.basename(s)[:-3] + ".o") for s in srcs]
    if not force and not _stale(lib):
        return lib
    nvcc = os.environ.get("NVCC", "nvcc")

    def comp(pair):
        s, o = pair
        cmd = [nvcc, *ARCH, *flags, "-c", s, "-o", o]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (s, r.stdout, r.stderr))
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return o

    with ThreadPoolExecutor(max_workers=max(1, len(srcs))) as ex:
        list(ex.map(comp, zip(srcs, objs)))
    tmp = lib + ".tmp%d" % os.getpid()
    subprocess.check_call([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"])
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv))
