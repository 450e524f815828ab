"""Build libhx.so in-tree with nvcc for sm_103a.

Each (degree, precision) kernel unit is hx_ops.cu compiled with -DHX_P and
-DHX_UNIT_F32; the units, the vector kernels, the C-ABI layer and the host-only
load vectors are compiled in parallel and linked into
paper_2408_12479_gb300/_lib/libhx.so.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INC = os.path.join(ROOT, "include")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libhx.so")
DEGREES = (1, 2, 3, 4, 5, 6)
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    p = shutil.which("nvcc")
    if p:
        return p
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found")


def _sources_digest(extra: str) -> str:
    h = hashlib.sha256(extra.encode())
    for d in (CSRC, INC):
        for f in sorted(os.listdir(d)):
            if f.endswith((".cu", ".h", ".cuh", ".cpp")):
                with open(os.path.join(d, f), "rb") as fh:
                    h.update(f.encode())
                    h.update(fh.read())
    return h.hexdigest()


def strip_comments(src: str) -> str:
    """C/C++/CUDA source with every comment replaced by one space and every
    run of whitespace collapsed to one space; string and character literals
    are kept as they are."""
    out = []
    i, n = 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
            out.append(" ")
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def kernel_sources() -> set:
    """The CUDA translation units (csrc/*.cu) and every header they include,
    directly or not: the code that defines, launches and feeds the kernels.
    Host-only units that no kernel unit includes are not part of it."""
    import re
    inc = re.compile(r'\s*#\s*include\s+"([^"]+)"')
    stack = [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC)) if f.endswith(".cu")]
    seen = set()
    while stack:
        path = os.path.normpath(stack.pop())
        if path in seen:
            continue
        seen.add(path)
        with open(path, encoding="utf-8") as fh:
            for line in fh:
                m = inc.match(line)
                if m:
                    for d in (os.path.dirname(path), CSRC, INC):
                        cand = os.path.join(d, m.group(1))
                        if os.path.exists(cand):
                            stack.append(cand)
                            break
    return seen


def kernel_digest() -> str:
    """Digest of kernel_sources() with comments and formatting removed:
    profile summaries record it so that their counters can be matched to the
    code, and an edit that changes only comments leaves it as it was."""
    src = kernel_sources()
    h = hashlib.sha256()
    for d in (CSRC, INC):
        for f in sorted(os.listdir(d)):
            path = os.path.normpath(os.path.join(d, f))
            if path in src:
                with open(path, encoding="utf-8") as fh:
                    h.update(f.encode())
                    h.update(strip_comments(fh.read()).encode())
    return h.hexdigest()


def build(force: bool = False, jobs: int | None = None, verbose: bool = False) -> str:
    nvcc = _nvcc()
    os.makedirs(LIBDIR, exist_ok=True)
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INC, "-I" + CSRC,
                    "--expt-relaxed-constexpr", "-diag-suppress", "177"]
    digest = _sources_digest(" ".join(flags) + nvcc)
    stamp = os.path.join(LIBDIR, "libhx.sha256")
    if not force and os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == digest:
        return LIB
    objdir = os.path.join(LIBDIR, "obj")
    os.makedirs(objdir, exist_ok=True)
    jobs_list = []
    for p in DEGREES:
        for f32 in (0, 1):
            obj = os.path.join(objdir, f"hx_ops_p{p}_{'f32' if f32 else 'f64'}.o")
            jobs_list.append([nvcc] + flags + [f"-DHX_P={p}", f"-DHX_UNIT_F32={f32}", "-c",
                                               os.path.join(CSRC, "hx_ops.cu"), "-o", obj])
    for f32 in (0, 1):
        jobs_list.append([nvcc] + flags + [f"-DHX_UNIT_F32={f32}", "-c", os.path.join(CSRC, "hx_batch.cu"), "-o",
                                           os.path.join(objdir, f"hx_batch_{'f32' if f32 else 'f64'}.o")])
    for name in ("hx_vec", "hx_api"):
        jobs_list.append([nvcc] + flags + ["-c", os.path.join(CSRC, name + ".cu"), "-o",
                                           os.path.join(objdir, name + ".o")])
    # host-only C++ (load vectors): no device code, so no -gencode
    jobs_list.append([nvcc, "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INC, "-c",
                      os.path.join(CSRC, "hx_loads.cpp"), "-o", os.path.join(objdir, "hx_loads.o")])
    # longest units first (the batch units include every degree)
    jobs_list.sort(key=lambda c: -(99 if any("hx_batch" in a for a in c) else
                                   int(next((a.split("=")[1] for a in c if a.startswith("-DHX_P=")), "0"))))
    n = jobs or max(1, min(len(jobs_list), os.cpu_count() or 4))

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose:
            sys.stderr.write(r.stderr)
        return cmd[-1]

    with cf.ThreadPoolExecutor(max_workers=n) as ex:
        objs = list(ex.map(run, jobs_list))
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"])
    os.replace(tmp, LIB)
    with open(stamp, "w") as fh:
        fh.write(digest)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
