"""Builds libqg.so in-tree with nvcc for sm_103a (GB300).

    python -m paper_2310_06650_gb300.build

The translation units compile in parallel; the shared library lands in
paper_2310_06650_gb300/_build/ (git-ignored).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libqg.so")
SOURCES = ["qg_kernels.cu", "qg_host.cu", "qg_mlp.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found; libqg needs the CUDA 13 toolkit")
    return cand


def _newest_source_mtime() -> float:
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    paths.append(os.path.join(os.path.dirname(HERE), "include", "qg.h"))
    paths.append(os.path.abspath(__file__))
    return max(os.path.getmtime(p) for p in paths if os.path.exists(p))


def checked_source(text: str) -> str:
    """The index-checked form of qg_kernels.cu: every d.<array>[i] becomes qg_at(d.<array>, i, __LINE__)
    (nested accesses too); no line breaks are added, so __LINE__ stays the original line."""
    out, i, n = [], 0, len(text)
    ident = set("abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ0123456789_.")
    while i < n:
        j = text.find("d.", i)
        if j < 0:
            out.append(text[i:])
            break
        k = j + 2
        while k < n and (text[k].isalnum() or text[k] == "_"):
            k += 1
        if (j > 0 and text[j - 1] in ident) or k == j + 2 or k >= n or text[k] != "[":
            out.append(text[i:j + 2])
            i = j + 2
            continue
        depth, e = 0, k
        while e < n:  # the matching bracket
            if text[e] == "[":
                depth += 1
            elif text[e] == "]":
                depth -= 1
                if depth == 0:
                    break
            e += 1
        out.append(text[i:j])
        out.append(f"qg_at({text[j:k]}, (long long)({checked_source(text[k + 1:e])}), __LINE__)")
        i = e + 1
    return "".join(out)


def build(force: bool = False, verbose: bool = False, check_bounds: bool = False) -> str:
    """Compile (if stale) and return the path of libqg.so.  check_bounds: the index-checked library
    (QG_CHECK_BOUNDS, every d.<array>[i] of the stage kernels checked) in _build/checked/."""
    out = os.path.join(OUT, "checked") if check_bounds else OUT
    lib = os.path.join(out, "libqg.so")
    os.makedirs(out, exist_ok=True)
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _newest_source_mtime():
        return lib
    nvcc = _nvcc()
    extra = ["-DQG_CHECK_BOUNDS", "-I", CSRC] if check_bounds else []

    def compile_one(src):
        obj = os.path.join(out, os.path.splitext(src)[0] + ".o")
        path = os.path.join(CSRC, src)
        if check_bounds and src == "qg_kernels.cu":
            with open(path) as f:
                text = f.read()
            path = os.path.join(out, src)
            with open(path, "w") as f:
                f.write(f'#line 1 "{os.path.join(CSRC, src)}"\n' + checked_source(text))
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", path, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stdout.write(r.stdout + r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + ".tmp"
    r = subprocess.run([nvcc, *ARCH, "-shared", *objs, "-o", tmp, "-lcudart"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, check_bounds="--check-bounds" in sys.argv))
