"""Compile generated kernels and call them.

CUDA: the kernel plus an ``extern "C"`` launcher are compiled by nvcc for
sm_103a into a shared object (cached by source hash under codegen/_build) and
called through ctypes with device pointers. C: the loop nest is compiled by
the system C compiler (no contraction of * and +) and called with host
arrays; the outermost parallel loop may run on OpenMP threads, since a
parallel loop's iterations write disjoint parts of its output.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import shutil
import subprocess
import threading

from . import emit as E
from . import phrase as P

HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.path.join(HERE, "_build")
_lock = threading.Lock()
NP_DTYPE = {"float": "float32", "int": "int32", "long long": "int64"}


def _nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: generated CUDA kernels need the CUDA toolkit")


_locks = {}


def _lock_for(key: str) -> threading.Lock:
    with _lock:
        return _locks.setdefault(key, threading.Lock())


def _build(src: str, suffix: str, cmd_for) -> str:
    """Compile src once into the cache (one lock per source, so that different
    kernels may compile on several threads at once)."""
    h = hashlib.sha256(src.encode()).hexdigest()[:20]
    d = os.path.join(CACHE, h)
    lib = os.path.join(d, "lib.so")
    with _lock_for(h):
        if not os.path.exists(lib):
            os.makedirs(d, exist_ok=True)
            path = os.path.join(d, "src" + suffix)
            with open(path, "w") as f:
                f.write(src)
            tmp = lib + f".tmp{os.getpid()}"
            r = subprocess.run(cmd_for(path, tmp), capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"compiling generated code failed:\n{r.stdout}\n{r.stderr}\n{src}")
            os.replace(tmp, lib)
    return lib


def cuda_source(gen: dict) -> str:
    name = gen["kernel"]
    params = gen["params"]
    casts = []
    for k, (pname, ct, _, role) in enumerate(params):
        q = "const " if role == "in" else ""
        casts.append(f"({q}{ct} *)a{k}")
    args = ", ".join(f"void *a{k}" for k in range(len(params)))
    return (
        "#include <cuda_runtime.h>\n\n"
        f"{gen['source']}\n"
        f"extern \"C\" int launch_{name}({args}, int grid, int block, void *stream) {{\n"
        f"  {name}<<<grid, block, 0, (cudaStream_t)stream>>>({', '.join(casts)});\n"
        "  return (int)cudaGetLastError();\n"
        "}\n")


class CudaKernel:
    """A generated CUDA kernel: run(*arrays, grid=, block=) with torch tensors
    (inputs, then the output, then the hoisted temporaries, as in .params)."""

    def __init__(self, gen: dict):
        self.gen = gen
        self.source = cuda_source(gen)
        lib = _build(self.source, ".cu", lambda src, out: [
            _nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-fmad=false", "-shared",
            "-Xcompiler", "-fPIC", "-lineinfo", "-o", out, src])
        self.lib = ctypes.CDLL(lib)
        self.fn = getattr(self.lib, "launch_" + gen["kernel"])
        self.fn.restype = ctypes.c_int
        self.fn.argtypes = [ctypes.c_void_p] * len(gen["params"]) + [ctypes.c_int, ctypes.c_int, ctypes.c_void_p]

    @property
    def params(self):
        return self.gen["params"]

    @property
    def uses_warps(self) -> bool:
        """The kernel has warp or lane loops (shuffles need all 32 lanes of a warp)."""
        return any(lvl in ("warp", "lane") for lvl, _ in _parallel_loops(self.gen["comm"]))

    def default_launch(self, sms: int = 152):
        """(grid, block) from the loop nest: the workgroup loop's trip count (or
        the global loop's) and the local loop's trip count, within limits."""
        wg = gl = loc = warp = None
        for lvl, n in _parallel_loops(self.gen["comm"]):
            if lvl == "workgroup" and wg is None:
                wg = n
            elif lvl == "local" and loc is None:
                loc = n
            elif lvl == "warp" and warp is None:
                warp = n
            elif lvl == "global" and gl is None:
                gl = n
        block = min(loc, 1024) if loc else (min(32 * warp, 1024) if warp else 256)
        if self.uses_warps:
            block = max(32, block // 32 * 32)
        if wg is not None:
            grid = max(1, min(wg, 65535 * 32))
        elif gl is not None:
            grid = max(1, min(-(-gl // block), sms * 8))
        else:
            grid, block = 1, 1
        return grid, block

    def run(self, *arrays, grid=None, block=None, stream=None):
        import torch

        if len(arrays) != len(self.params):
            raise ValueError(f"{self.gen['kernel']} takes {len(self.params)} arrays "
                             f"({', '.join(p[0] for p in self.params)})")
        for a, (pname, ct, count, _) in zip(arrays, self.params):
            if not (isinstance(a, torch.Tensor) and a.is_cuda and a.is_contiguous()):
                raise ValueError(f"{pname}: a contiguous CUDA tensor is required")
            if str(a.dtype).replace("torch.", "") != NP_DTYPE[ct] or a.numel() < count:
                raise ValueError(f"{pname}: need {count} x {NP_DTYPE[ct]}, got {a.numel()} x {a.dtype}")
        g0, b0 = self.default_launch()
        grid, block = grid or g0, block or b0
        if not (1 <= block <= 1024 and grid >= 1):
            raise ValueError("grid >= 1 and 1 <= block <= 1024")
        if self.uses_warps and block % 32:
            raise ValueError("a kernel with warp or lane loops needs whole warps: block a multiple of 32")
        s = stream or torch.cuda.current_stream()
        rc = self.fn(*[ctypes.c_void_p(a.data_ptr()) for a in arrays], int(grid), int(block),
                     ctypes.c_void_p(s.cuda_stream))
        if rc != 0:
            raise RuntimeError(f"launch of {self.gen['kernel']} failed: CUDA error {rc}")

    def temps_like(self, device="cuda"):
        """Zero-filled hoisted temporaries for run()."""
        import torch

        return [torch.zeros(count, dtype=getattr(torch, NP_DTYPE[ct]), device=device)
                for (_, ct, count, role) in self.params if role == "temp"]


class CFunction:
    """The same loop nest compiled as C for the host (run with numpy arrays)."""

    def __init__(self, gen: dict, openmp: bool = False):
        self.gen = gen
        src = gen["source"]
        if openmp:
            src = _omp_outer(src)
        self.source = src
        flags = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11"]
        if openmp:
            flags.append("-fopenmp")
        cc = os.environ.get("CC", "gcc")
        self.lib = ctypes.CDLL(_build(src, ".c", lambda s, out: [cc, *flags, "-o", out, s, "-lm"]))
        self.fn = getattr(self.lib, gen["kernel"])
        self.fn.restype = None
        self.fn.argtypes = [ctypes.c_void_p] * len(gen["params"])

    @property
    def params(self):
        return self.gen["params"]

    def run(self, *arrays):
        import numpy as np

        if len(arrays) != len(self.params):
            raise ValueError(f"{self.gen['kernel']} takes {len(self.params)} arrays")
        for a, (pname, ct, count, _) in zip(arrays, self.params):
            if not (isinstance(a, np.ndarray) and a.flags.c_contiguous and a.dtype == np.dtype(NP_DTYPE[ct])
                    and a.size >= count):
                raise ValueError(f"{pname}: need a contiguous {count} x {NP_DTYPE[ct]} array")
        self.fn(*[a.ctypes.data_as(ctypes.c_void_p) for a in arrays])

    def temps_like(self):
        import numpy as np

        return [np.zeros(count, dtype=NP_DTYPE[ct]) for (_, ct, count, role) in self.params if role == "temp"]


def _omp_outer(src: str) -> str:
    """Run the outermost parallel loops (work-group or global maps, marked by
    the emitter) on OpenMP threads; sequential loops, such as a fold at the top
    of a program or the second level after the work-group loop, stay on one."""
    return src.replace(E.OMP_MARK, "#pragma omp parallel for schedule(static)")


def _parallel_loops(c, out=None):
    from . import translate as T

    out = [] if out is None else out
    if isinstance(c, T.For):
        if c.level != "seq":
            out.append((c.level, c.n))
        _parallel_loops(c.body, out)
    elif isinstance(c, T.Seq):
        for x in c.cs:
            _parallel_loops(x, out)
    elif isinstance(c, T.New):
        _parallel_loops(c.body, out)
    elif isinstance(c, T.TreeReduce):
        out.append(("lane", c.buf.type.n))
        _parallel_loops(c.fill, out)
    elif isinstance(c, T.LastBlock):
        _parallel_loops(c.body, out)
    return out


def compile_cuda(name: str, expr: P.Phrase, inputs: list, unroll: int = 1) -> CudaKernel:
    return CudaKernel(E.generate(name, expr, inputs, "cuda", unroll=unroll))


def compile_c(name: str, expr: P.Phrase, inputs: list, openmp: bool = False) -> CFunction:
    return CFunction(E.generate(name, expr, inputs, "c"), openmp=openmp)
