"""Build libqmc_gb300.so (and its checked build libqmc_gb300_checked.so) in-tree: one
nvcc process per translation unit (all in parallel), sm_103a only, then a shared link
against the shared CUDA runtime."""
from __future__ import annotations

import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libqmc_gb300.so")
HEADER = os.path.join(ROOT, "include", "qmc.h")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    raise RuntimeError("nvcc not found")


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def code_only(text: str) -> str:
    """C/C++ source without its comments and blank lines, each line stripped of
    trailing blanks: what a comment-only edit leaves unchanged."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c in "\"'":  # a string or character literal, copied whole
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    lines = (line.rstrip() for line in "".join(out).split("\n"))
    return "\n".join(line for line in lines if line)


def source_digest(files: list[str] | None = None) -> str:
    """Short hash of the code of the given csrc files (default: every CUDA source
    and header), comments left out; ties a profile figure to the code of the
    kernel it was taken from."""
    import hashlib

    h = hashlib.sha256()
    if files:
        deps = [os.path.join(CSRC, f) for f in files]
    else:
        deps = sorted(sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")))
        deps.append(HEADER)
    for d in deps:
        h.update(os.path.basename(d).encode())
        with open(d, encoding="utf-8") as f:
            h.update(code_only(f.read()).encode())
    return h.hexdigest()[:12]


LIB_CHECKED = os.path.join(PKG, "libqmc_gb300_checked.so")


def _deps() -> list[str]:
    return sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + [HEADER]


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in _deps())


def _compile(build_dir: str, flags: list[str], verbose: bool):
    """Starts one nvcc per translation unit; returns (objects, [(source, process)])."""
    os.makedirs(build_dir, exist_ok=True)
    procs, objs = [], []
    for src in sources():
        obj = os.path.join(build_dir, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        cmd = [_nvcc(), *flags, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    return objs, procs


def build(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None,
          checked: bool = True) -> str:
    """Compile every CUDA source of the package into libqmc_gb300.so and, with `checked`,
    into the checked build libqmc_gb300_checked.so (-DQMC_CHECKED=1: bounds-tested stores),
    all translation units of both in parallel; returns the normal library's path."""
    flags = ["-O3", "-std=c++17", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
             "-I", os.path.join(ROOT, "include"), *(extra_flags or [])]
    jobs = []
    if force or _stale(LIB):
        jobs.append((LIB, *_compile(BUILD, flags, verbose)))
    if checked and (force or _stale(LIB_CHECKED)):
        jobs.append((LIB_CHECKED, *_compile(BUILD + "_checked", flags + ["-DQMC_CHECKED=1"], verbose)))
    failed = []
    for _, _, procs in jobs:
        for src, p in procs:
            out, _ = p.communicate()
            if p.returncode != 0:
                failed.append(f"{src}:\n{out.decode(errors='replace')}")
            elif verbose and out:
                print(out.decode(errors="replace"), file=sys.stderr)
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(failed))
    for lib, objs, _ in jobs:
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.check_call([_nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs])
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
