"""Stage III (Section 4.3): the loop nest becomes CUDA C (or plain C).

Views are resolved into index arithmetic on the arrays they read: an access
path (a list of index and projection steps, innermost last) is pushed through
``split``, ``join``, ``transpose``, ``zip`` and the projections until it
reaches an input or a temporary, where it becomes a row-major offset. Writes
through acceptors are resolved the same way. Loops map to the hierarchy:

    global     for (i = blockIdx.x*blockDim.x + threadIdx.x; i < n; i += gridDim.x*blockDim.x)
    workgroup  for (i = blockIdx.x; i < n; i += gridDim.x)
    local      for (i = threadIdx.x; i < n; i += blockDim.x)
    warp       for (i = threadIdx.x / 32; i < n; i += blockDim.x / 32)
    lane       for (i = threadIdx.x % 32; i < n; i += 32)
    seq        for (i = 0; i < n; ++i)

A statement outside every parallel loop runs in one thread (thread 0 of block
0, thread 0 of the workgroup when it sits in a workgroup loop only, lane 0
when it sits in a warp loop). A lane tree keeps element l in lane l's
register and combines with warp shuffles (``__shfl_down_sync`` by L/2, L/4,
.., 1: lane l adds lane l + h's value, the halving tree); the C backend keeps
the elements in an array and runs the same halving loops. The second level
runs in the last block: after a block barrier, thread 0 fences the block's
writes and takes a ticket (atomicAdd on a counter); the block that draws the
last one fences again,
reads the parts through L2 (``__ldcg``), computes the second level and puts
the counter back to zero -- no block ever waits for another. Where
a temporary in local or global memory is in scope, block barriers separate a
local loop from the statements before and after it and end every iteration of
a loop that contains a local loop, so no thread reads what another has not
finished writing, nor overwrites what another still reads (writes through the
output acceptor go to disjoint places and are never read back). Temporaries:
private ones are C variables (arrays of the loop body), local ones shared
arrays, global ones slices of a hoisted buffer, one slice per iteration of the
parallel loops around them (Section 6.4). In the C backend every loop is
sequential.

Floating-point + and * are emitted as separately rounded operations
(``__fadd_rn`` / ``__fmul_rn`` in CUDA, plain float arithmetic compiled
without contraction in C), so the generated code evaluates exactly the tree
the phrase denotes.
"""
from __future__ import annotations

import math

from . import phrase as P
from . import translate as T

CTYPE = {"f32": "float", "i32": "int", "i64": "long long"}
VTYPE = {2: "float2", 4: "float4"}
LANES = "xyzw"


def ctype(t) -> str:
    """C type of a number or vector."""
    if isinstance(t, P.VecT):
        return VTYPE[t.n]
    return CTYPE[t.dtype]


# Lane-wise vector arithmetic, each lane rounded separately.
CUDA_PRELUDE = """#define DPIA_V4(name, op) __device__ __forceinline__ float4 name(float4 a, float4 b) { \\
  return make_float4(op(a.x, b.x), op(a.y, b.y), op(a.z, b.z), op(a.w, b.w)); }
#define DPIA_V2(name, op) __device__ __forceinline__ float2 name(float2 a, float2 b) { \\
  return make_float2(op(a.x, b.x), op(a.y, b.y)); }
DPIA_V4(dpia_vadd4, __fadd_rn) DPIA_V4(dpia_vsub4, __fsub_rn) DPIA_V4(dpia_vmul4, __fmul_rn)
DPIA_V2(dpia_vadd2, __fadd_rn) DPIA_V2(dpia_vsub2, __fsub_rn) DPIA_V2(dpia_vmul2, __fmul_rn)
__device__ __forceinline__ float dpia_lane4(float4 v, long long l) {
  return l == 0 ? v.x : l == 1 ? v.y : l == 2 ? v.z : v.w; }
__device__ __forceinline__ float dpia_lane2(float2 v, long long l) { return l == 0 ? v.x : v.y; }
__device__ __forceinline__ float4 dpia_vabs4(float4 a) { return make_float4(fabsf(a.x), fabsf(a.y), fabsf(a.z), fabsf(a.w)); }
__device__ __forceinline__ float2 dpia_vabs2(float2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }
__device__ __forceinline__ float4 dpia_splat4(float v) { return make_float4(v, v, v, v); }
__device__ __forceinline__ float2 dpia_splat2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float4 dpia_vfma4(float4 a, float4 b, float4 c) {
  return make_float4(__fmaf_rn(a.x, b.x, c.x), __fmaf_rn(a.y, b.y, c.y), __fmaf_rn(a.z, b.z, c.z),
                     __fmaf_rn(a.w, b.w, c.w)); }
__device__ __forceinline__ float2 dpia_vfma2(float2 a, float2 b, float2 c) {
  return make_float2(__fmaf_rn(a.x, b.x, c.x), __fmaf_rn(a.y, b.y, c.y)); }
"""

THREADED = ("local", "warp", "lane")  # levels whose loops spread over the threads of a block
OMP_MARK = "/* dpia: outermost parallel loop */"

C_PRELUDE = """#include <math.h>
typedef struct { float x, y, z, w; } float4;
typedef struct { float x, y; } float2;
static inline float4 make_float4(float x, float y, float z, float w) { float4 v = {x, y, z, w}; return v; }
static inline float2 make_float2(float x, float y) { float2 v = {x, y}; return v; }
static inline float f_add(float a, float b) { return a + b; }
static inline float f_sub(float a, float b) { return a - b; }
static inline float f_mul(float a, float b) { return a * b; }
#define DPIA_V4(name, op) static inline float4 name(float4 a, float4 b) { \\
  return make_float4(op(a.x, b.x), op(a.y, b.y), op(a.z, b.z), op(a.w, b.w)); }
#define DPIA_V2(name, op) static inline float2 name(float2 a, float2 b) { \\
  return make_float2(op(a.x, b.x), op(a.y, b.y)); }
DPIA_V4(dpia_vadd4, f_add) DPIA_V4(dpia_vsub4, f_sub) DPIA_V4(dpia_vmul4, f_mul)
DPIA_V2(dpia_vadd2, f_add) DPIA_V2(dpia_vsub2, f_sub) DPIA_V2(dpia_vmul2, f_mul)
static inline float dpia_lane4(float4 v, long long l) { return l == 0 ? v.x : l == 1 ? v.y : l == 2 ? v.z : v.w; }
static inline float dpia_lane2(float2 v, long long l) { return l == 0 ? v.x : v.y; }
static inline float4 dpia_vabs4(float4 a) { return make_float4(fabsf(a.x), fabsf(a.y), fabsf(a.z), fabsf(a.w)); }
static inline float2 dpia_vabs2(float2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }
static inline float4 dpia_splat4(float v) { return make_float4(v, v, v, v); }
static inline float2 dpia_splat2(float v) { return make_float2(v, v); }
static inline float4 dpia_vfma4(float4 a, float4 b, float4 c) {
  return make_float4(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y), fmaf(a.z, b.z, c.z), fmaf(a.w, b.w, c.w)); }
static inline float2 dpia_vfma2(float2 a, float2 b, float2 c) {
  return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y)); }
"""


def _acc_root(a):
    while not isinstance(a, T.AOut):
        a = a.acc
    return a


def _reads_lane_or_private_element(e) -> bool:
    """The expression reads an element of a private array temporary, or a lane of
    a vector (unrolled, a lane index is a constant: a register, not a select)."""
    if isinstance(e, P.Ident):
        return e.temp == "private" and isinstance(e.type, P.Arr)
    if isinstance(e, P.Lanes):
        return True
    return any(_reads_lane_or_private_element(x) for x in e.children())


def _indexes_registers(c) -> bool:
    """The command writes or reads an element of a private array temporary, or
    reads a lane of a vector: indices that unrolling turns into constants."""
    if isinstance(c, T.Assign):
        r = _acc_root(c.acc)
        return (r.temp is not None and r.temp.space == "private" and isinstance(r.temp.type, P.Arr)) or \
            _reads_lane_or_private_element(c.e)
    if isinstance(c, T.Seq):
        return any(_indexes_registers(x) for x in c.cs)
    if isinstance(c, (T.New, T.For)):
        return _indexes_registers(c.body)
    return False


def divisible(i, V: int) -> bool:
    """True if the index expression is a multiple of V for every value of its variables."""
    if isinstance(i, T.IConst):
        return i.v % V == 0
    if isinstance(i, T.IOp):
        if i.op == "+":
            return divisible(i.a, V) and divisible(i.b, V)
        if i.op == "*":
            return divisible(i.a, V) or divisible(i.b, V)
    return False


class EmitError(Exception):
    pass


def render_index(i) -> str:
    if isinstance(i, T.IConst):
        return str(i.v)
    if isinstance(i, T.IVar):
        return i.name
    if isinstance(i, T.IOp):
        return f"({render_index(i.a)} {i.op} {render_index(i.b)})"
    raise EmitError(f"bad index {i!r}")


def dims(t) -> list:
    d = []
    while isinstance(t, P.Arr):
        d.append(t.n)
        t = t.elem
    return d


def linear(idx: list, shape: list):
    """Row-major offset of idx (len(idx) == len(shape))."""
    if len(idx) != len(shape):
        raise EmitError(f"access with {len(idx)} indices into an array of rank {len(shape)}")
    off = T.IConst(0)
    for i, n in zip(idx, shape):
        off = T.iadd(T.imul(off, n), i)
    return off


class Emitter:
    in_last = False  # emitting the last block's second level: parts are read through L2

    def __init__(self, backend: str, inputs: list, out: T.AOut, temps: list, unroll: int = 1):
        if backend not in ("cuda", "c"):
            raise EmitError(f"unknown backend {backend}")
        self.backend = backend
        self.unroll = unroll
        self.inputs = {p.name: p for p in inputs}
        self.out = out
        self.temps = {t.name: t for t in temps}
        self.lines = []
        self.shared = []
        self.private_ctx = {}  # private temp name -> parallel depth where declared
        # per loop scope: are temporaries shared between the block's threads in
        # play (then barriers separate thread-level loops from what follows)?
        self.sync = [False]

    # -- reads ----------------------------------------------------------------

    def access(self, e: P.Phrase, path: list) -> str:
        """C expression for the number reached from e by path (steps applied in order)."""
        if isinstance(e, P.Idx):
            return self.access(e.e, [("i", e.i)] + path)
        if isinstance(e, P.Proj):
            return self.access(e.e, [("p", e.k)] + path)
        if isinstance(e, P.Zip):
            if len(path) < 2 or path[0][0] != "i" or path[1][0] != "p":
                raise EmitError("a zipped pair must be indexed and projected")
            return self.access(e.b if path[1][1] else e.a, [path[0]] + path[2:])
        if isinstance(e, P.Pair):
            if not path or path[0][0] != "p":
                raise EmitError("a pair must be projected")
            return self.access(e.b if path[0][1] else e.a, path[1:])
        if isinstance(e, P.Split):
            if len(path) < 2 or path[0][0] != "i" or path[1][0] != "i":
                raise EmitError("split read without two indices")
            return self.access(e.e, [("i", T.iadd(T.imul(path[0][1], e.n), path[1][1]))] + path[2:])
        if isinstance(e, P.Join):
            m = e.e.type.elem.n
            k = path[0][1]
            return self.access(e.e, [("i", T.idiv(k, m)), ("i", T.imod(k, m))] + path[1:])
        if isinstance(e, P.Transpose):
            if len(path) < 2:
                raise EmitError("transpose read without two indices")
            return self.access(e.e, [path[1], path[0]] + path[2:])
        if isinstance(e, P.To):
            return self.access(e.e, path)
        if isinstance(e, P.AsVector):
            if len(path) != 1 or path[0][0] != "i":
                raise EmitError("asVector read must select one whole vector")
            base, off = self.locate(e.e, [("i", T.imul(path[0][1], e.n))])
            if not divisible(off, e.n):
                raise EmitError(f"asVector {e.n} access at offset {render_index(off)} is not provably aligned")
            q = "const " if base in self.inputs else ""
            return f"reinterpret_cast<{q}{VTYPE[e.n]} *>({base})[{render_index(T.idiv(off, e.n))}]" \
                if self.backend == "cuda" else f"(({q}{VTYPE[e.n]} *){base})[{render_index(T.idiv(off, e.n))}]"
        if isinstance(e, P.AsScalar):
            V = e.e.type.elem.n
            k = path[0][1]
            v = self.access(e.e, [("i", T.idiv(k, V))])
            lane = T.imod(k, V)
            if isinstance(lane, T.IConst):
                return f"({v}).{LANES[lane.v]}"
            return f"dpia_lane{V}({v}, {render_index(lane)})"
        if isinstance(e, P.Lanes):
            if isinstance(e.e.type, P.PairT):  # lane v of a pair of vectors: component k's lane v
                V = e.e.type.a.n
                if len(path) != 2 or path[0][0] != "i" or path[1][0] != "p":
                    raise EmitError("lanes of a pair: select one lane, then a component")
                v = self.access(e.e, [path[1]])
                path = path[:1]
            else:
                V = e.e.type.n
                if len(path) != 1 or path[0][0] != "i":
                    raise EmitError("lanes read must select one lane")
                v = self.access(e.e, [])
            lane = path[0][1]
            if isinstance(lane, T.IConst):
                return f"({v}).{LANES[lane.v]}"
            return f"dpia_lane{V}({v}, {render_index(lane)})"
        if isinstance(e, Shuffle):
            return f"__shfl_down_sync(0xffffffffu, {self.access(e.e, path)}, {e.offset})"
        if isinstance(e, P.Lit):
            if isinstance(e.type, P.Arr):  # every element of an array literal is its value
                return self.literal(P.Lit(e.value, P.base_elem(e.type)))
            return self.literal(e)
        if isinstance(e, P.Bin):
            if path:
                raise EmitError("index into a number")
            a, b = self.access(e.a, []), self.access(e.b, [])
            return self.binop(e.op, a, b, e.type)
        if isinstance(e, P.Fma):
            if path:
                raise EmitError("index into a number")
            a, b, c = self.access(e.a, []), self.access(e.b, []), self.access(e.c, [])
            if isinstance(e.type, P.VecT):
                return f"dpia_vfma{e.type.n}({a}, {b}, {c})"
            return f"__fmaf_rn({a}, {b}, {c})" if self.backend == "cuda" else f"fmaf({a}, {b}, {c})"
        if isinstance(e, P.Splat):
            if path:  # a lane of the vector: the number itself
                return self.access(e.a, [])
            return f"dpia_splat{e.n}({self.access(e.a, [])})"
        if isinstance(e, P.Abs):
            if isinstance(e.type, P.VecT):
                return f"dpia_vabs{e.type.n}({self.access(e.a, [])})"
            return f"fabsf({self.access(e.a, [])})"
        if isinstance(e, P.Ident):
            return self.base_read(e, path)
        raise EmitError(f"cannot read a {type(e).__name__} (did a map or reduce escape translation?)")

    def locate(self, e: P.Phrase, path: list):
        """(array name, offset) of the element of e reached by path. Only views
        that keep an array's elements adjacent in memory (index, split, join)
        may lie between asVector and the input it reads."""
        while True:
            if isinstance(e, P.Idx):
                path = [("i", e.i)] + path
                e = e.e
            elif isinstance(e, P.Split):
                path = [("i", T.iadd(T.imul(path[0][1], e.n), path[1][1]))] + path[2:]
                e = e.e
            elif isinstance(e, P.Join):
                m = e.e.type.elem.n
                k = path[0][1]
                path = [("i", T.idiv(k, m)), ("i", T.imod(k, m))] + path[1:]
                e = e.e
            elif isinstance(e, P.Transpose):
                # neighbours of a transposed array are a row apart in memory
                raise EmitError("asVector of a transposed array: its lanes are not adjacent in memory")
            elif isinstance(e, P.To):
                e = e.e
            elif isinstance(e, P.Ident):
                if e.temp is not None or e.name not in self.inputs:
                    raise EmitError("asVector reads kernel inputs only")
                return e.name, linear([s_[1] for s_ in path], dims(e.type))
            else:
                raise EmitError(f"asVector of a {type(e).__name__}")

    def base_read(self, e: P.Ident, path: list) -> str:
        if e.temp is not None and isinstance(e.type, P.PairT):
            if len(path) != 1 or path[0][0] != "p":
                raise EmitError("a pair temporary is read one component at a time")
            return f"{e.name}_{path[0][1]}"
        if e.temp is not None and isinstance(P.base_elem(e.type), P.PairT) and path and path[-1][0] == "p":
            # a component of an element of an array of pairs
            if any(s[0] != "i" for s in path[:-1]):
                raise EmitError("an array of pairs is indexed, then projected")
            ref = self.temp_pair_ref(self.temps[e.name], [s[1] for s in path[:-1]], path[-1][1])
            if self.in_last and self.temps[e.name].space == "global" and self.backend == "cuda":
                return f"__ldcg(&{ref})"
            return ref
        idx = [s[1] for s in path]
        if any(s[0] != "i" for s in path):
            raise EmitError("projection of a non-pair")
        if e.temp is None:
            if e.name not in self.inputs:
                raise EmitError(f"unknown input {e.name}")
            if not idx:
                return e.name if isinstance(e.type, P.Num) else f"{e.name}[0]"
            return f"{e.name}[{render_index(linear(idx, dims(e.type)))}]"
        t = self.temps[e.name]
        ref = self.temp_ref(t, idx)
        if self.in_last and t.space == "global" and self.backend == "cuda":
            return f"__ldcg(&{ref})"  # written by other blocks: read through L2, not a stale L1 line
        return ref

    def temp_pair_ref(self, t: T.Temp, idx: list, k: int) -> str:
        """Component k of element idx of a temporary array of pairs (stored as
        two numbers per element); a lane tree's buffer of pairs is two registers."""
        if t.lanes and self.backend == "cuda":
            return f"{t.name}_{k}"
        shape = dims(t.type)
        off = T.iadd(T.imul(linear(idx, shape), 2), T.IConst(k)) if shape else T.IConst(k)
        if t.space == "global" and t.hoist:
            size = P.scalar_count(t.type)
            h = linear([v for v, _ in t.hoist], [n for _, n in t.hoist])
            off = T.iadd(T.imul(h, size), off)
        return f"{t.name}[{render_index(off)}]"

    def temp_ref(self, t: T.Temp, idx: list) -> str:
        shape = dims(t.type)
        if t.lanes and self.backend == "cuda":
            return t.name  # element l of a lane tree's buffer is lane l's register
        if t.space == "private":
            if not shape:
                return t.name
            return f"{t.name}[{render_index(linear(idx, shape))}]"
        off = linear(idx, shape) if shape else T.IConst(0)
        if t.space == "global" and t.hoist:
            size = P.scalar_count(t.type)
            h = linear([v for v, _ in t.hoist], [n for _, n in t.hoist])
            off = T.iadd(T.imul(h, size), off)
        return f"{t.name}[{render_index(off)}]"

    def literal(self, e: P.Lit) -> str:
        if isinstance(e.type, P.VecT):
            v = self.literal(P.Lit(e.value, e.type.num))
            return f"make_float{e.type.n}({', '.join([v] * e.type.n)})"
        if e.type.dtype == "f32":
            v = float(e.value)
            return f"{v!r}f" if v == v and abs(v) != float("inf") else "0.0f"
        return f"(({CTYPE[e.type.dtype]}){int(e.value)})"

    def binop(self, op, a, b, t) -> str:
        if isinstance(t, P.VecT):
            fn = {"+": "dpia_vadd", "-": "dpia_vsub", "*": "dpia_vmul"}[op]
            return f"{fn}{t.n}({a}, {b})"
        if t.dtype == "f32" and self.backend == "cuda":
            fn = {"+": "__fadd_rn", "-": "__fsub_rn", "*": "__fmul_rn"}[op]
            return f"{fn}({a}, {b})"
        return f"({a} {op} {b})"

    # -- writes ---------------------------------------------------------------

    def write(self, acc: T.Acc, path: list, proj=None) -> str:
        if isinstance(acc, T.AProj):
            return self.write(acc.acc, path, acc.k)
        if proj is not None:
            return self.write_pair(acc, path, proj)
        if isinstance(acc, T.AIdx):
            return self.write(acc.acc, [acc.i] + path)
        if isinstance(acc, T.ASplit):
            return self.write(acc.acc, [T.idiv(path[0], acc.n), T.imod(path[0], acc.n)] + path[1:])
        if isinstance(acc, T.AJoin):
            return self.write(acc.acc, [T.iadd(T.imul(path[0], acc.m), path[1])] + path[2:])
        if isinstance(acc, T.ATranspose):
            return self.write(acc.acc, [path[1], path[0]] + path[2:])
        if isinstance(acc, T.AAsScalar):
            # element j of the vector array is the V scalars at j*V of acc
            inner = acc.acc
            path2 = [T.imul(path[0], acc.V)] + path[1:]
            while not isinstance(inner, T.AOut):
                if isinstance(inner, T.AIdx):
                    path2 = [inner.i] + path2
                elif isinstance(inner, T.ASplit):
                    path2 = [T.idiv(path2[0], inner.n), T.imod(path2[0], inner.n)] + path2[1:]
                elif isinstance(inner, T.AJoin):
                    path2 = [T.iadd(T.imul(path2[0], inner.m), path2[1])] + path2[2:]
                else:
                    raise EmitError("asScalar output through a transposed acceptor")
                inner = inner.acc
            if inner.temp is not None:
                raise EmitError("asScalar into a temporary")
            off = linear(path2, dims(inner.type))
            if not divisible(off, acc.V):
                raise EmitError("asScalar store not provably aligned")
            vt = VTYPE[acc.V]
            cast = f"reinterpret_cast<{vt} *>({inner.name})" if self.backend == "cuda" else f"(({vt} *){inner.name})"
            return f"{cast}[{render_index(T.idiv(off, acc.V))}]"
        if isinstance(acc, T.AOut):
            if acc.temp is not None:
                return self.temp_ref(acc.temp, path)
            shape = dims(acc.type)
            if isinstance(P.base_elem(acc.type), P.VecT):
                vt = ctype(P.base_elem(acc.type))
                cast = f"reinterpret_cast<{vt} *>({acc.name})" if self.backend == "cuda" else f"(({vt} *){acc.name})"
                return f"{cast}[{render_index(linear(path, shape)) if shape else '0'}]"
            if not shape:
                return f"{acc.name}[0]"
            return f"{acc.name}[{render_index(linear(path, shape))}]"
        raise EmitError(f"unknown acceptor {type(acc).__name__}")

    def write_pair(self, acc: T.Acc, path: list, k: int) -> str:
        """Component k of the pair reached through acc by path."""
        while not isinstance(acc, T.AOut):
            if isinstance(acc, T.AIdx):
                path = [acc.i] + path
            elif isinstance(acc, T.ASplit):
                path = [T.idiv(path[0], acc.n), T.imod(path[0], acc.n)] + path[1:]
            elif isinstance(acc, T.AJoin):
                path = [T.iadd(T.imul(path[0], acc.m), path[1])] + path[2:]
            elif isinstance(acc, T.ATranspose):
                path = [path[1], path[0]] + path[2:]
            else:
                raise EmitError(f"pair component through a {type(acc).__name__}")
            acc = acc.acc
        if acc.temp is not None:
            if isinstance(acc.temp.type, P.PairT):  # a private pair: two variables
                return f"{acc.name}_{k}"
            return self.temp_pair_ref(acc.temp, path, k)
        if not isinstance(P.base_elem(acc.type), P.PairT):
            raise EmitError("pair component of a non-pair output")
        off = linear(path, dims(acc.type)) if dims(acc.type) else T.IConst(0)
        return f"{acc.name}[{render_index(T.iadd(T.imul(off, 2), T.IConst(k)))}]"

    # -- commands -------------------------------------------------------------

    def emit(self, c: T.Comm, ind: int, ctx: tuple):
        """ctx: the levels of the enclosing loops."""
        pad = "  " * ind
        if isinstance(c, T.Seq):
            uniform = _block_uniform(ctx)  # every thread of the block runs this code: a barrier may go here
            for k, x in enumerate(c.cs):
                local = self.backend == "cuda" and self.sync[-1] and uniform and _threaded(x)
                if local and k > 0:  # what the block's threads read was written by others
                    self.barrier(pad)
                self.emit(x, ind, ctx)
                if local and k + 1 < len(c.cs):  # and the other way round
                    self.barrier(pad)
            return
        if isinstance(c, T.New):
            t = c.temp
            if t.space != "private":
                self.sync[-1] = True
            if isinstance(P.base_elem(t.type), P.VecT) and t.space != "private":
                raise EmitError("vector temporaries are private only")
            if isinstance(t.type, P.PairT):
                if t.space != "private":
                    raise EmitError("pair temporaries are private scalars only")
                par = sum(1 for l in ctx if l != "seq")
                self.private_ctx[t.name] = (par, _per_thread(ctx))
                self.lines.append(f"{pad}{ctype(t.type.a)} {t.name}_0;")
                self.lines.append(f"{pad}{ctype(t.type.b)} {t.name}_1;")
                self.emit(c.body, ind, ctx)
                return
            if isinstance(P.base_elem(t.type), P.PairT) and t.space == "private":
                # an array of pairs: element j's components at 2j and 2j + 1
                par = sum(1 for l in ctx if l != "seq")
                self.private_ctx[t.name] = (par, _per_thread(ctx))
                self.lines.append(f"{pad}{ctype(P.base_num(t.type))} {t.name}[{P.scalar_count(t.type)}];")
                self.emit(c.body, ind, ctx)
                return
            if t.space == "private":
                ct = ctype(P.base_elem(t.type))
                shape = dims(t.type)
                par = sum(1 for l in ctx if l != "seq")
                self.private_ctx[t.name] = (par, _per_thread(ctx))
                if shape:  # one entry per element (a number or a vector)
                    self.lines.append(f"{pad}{ct} {t.name}[{math.prod(shape)}];")
                else:
                    self.lines.append(f"{pad}{ct} {t.name};")
            elif t.space == "local" and self.backend == "cuda":
                ct = CTYPE[P.base_num(t.type).dtype]
                if 4 * P.scalar_count(t.type) + sum(_shared_bytes(x) for x in self.shared) > 48 * 1024:
                    raise EmitError(f"local temporaries of more than 48 KiB per block ({t.name}: {t.type})")
                self.shared.append(f"  __shared__ {ct} {t.name}[{P.scalar_count(t.type)}];")
            elif t.space == "local":
                ct = CTYPE[P.base_num(t.type).dtype]
                self.lines.append(f"{pad}{ct} {t.name}[{P.scalar_count(t.type)}];")
            self.emit(c.body, ind, ctx)
            return
        if isinstance(c, T.Assign):
            self.check_private_reads(c.e, ctx)
            stmt = f"{self.write(c.acc, [])} = {self.access(c.e, [])};"
            self.lines.append(f"{pad}{self.guard(ctx)}{stmt}")
            return
        if isinstance(c, T.For):
            v, n = c.var.name, c.n
            if self.backend == "c" and c.level in ("workgroup", "global") and not ctx:
                # the outermost parallel loop: its iterations write disjoint places, so
                # the host build may run them on threads (each declares its own temporaries)
                self.lines.append(f"{pad}{OMP_MARK}")
            if self.backend == "c" or c.level == "seq":
                if c.level == "seq" and not self.has_parallel(c.body) and self.guard(ctx):
                    # a sequential loop outside the thread-level loops runs in one thread
                    self.lines.append(f"{pad}{self.guard(ctx).strip()} {{")
                    self.lines.append(f"{pad}  for (long long {v} = 0; {v} < {n}; ++{v}) {{")
                    self.emit(c.body, ind + 2, ctx + ("seq", "guarded"))
                    self.lines.append(f"{pad}  }}")
                    self.lines.append(f"{pad}}}")
                    return
                if self.backend == "cuda" and c.level == "seq" and n <= 16 and _indexes_registers(c.body):
                    # a short loop over a private array (e.g. a thread's tile of
                    # accumulators) or over a vector's lanes: unrolled whole, so that the
                    # array lives in registers and a lane is a register, not a select
                    self.lines.append(f"{pad}#pragma unroll")
                elif self.backend == "cuda" and self.unroll > 1 and c.level == "seq" and n > self.unroll:
                    # a sequential loop's iterations stay in order; unrolling only
                    # lets their loads be issued ahead of the dependent steps
                    self.lines.append(f"{pad}#pragma unroll {self.unroll}")
                self.lines.append(f"{pad}for (long long {v} = 0; {v} < {n}; ++{v}) {{")
            elif c.level == "workgroup":
                self.lines.append(f"{pad}for (long long {v} = blockIdx.x; {v} < {n}; {v} += gridDim.x) {{")
            elif c.level == "local":
                self.lines.append(f"{pad}for (long long {v} = threadIdx.x; {v} < {n}; {v} += blockDim.x) {{")
            elif c.level == "warp":
                self.lines.append(f"{pad}for (long long {v} = threadIdx.x >> 5; {v} < {n}; {v} += blockDim.x >> 5) {{")
            elif c.level == "lane":
                self.lines.append(f"{pad}for (long long {v} = threadIdx.x & 31; {v} < {n}; {v} += 32) {{")
            elif c.level == "global":
                self.lines.append(f"{pad}for (long long {v} = (long long)blockIdx.x * blockDim.x + threadIdx.x; "
                                  f"{v} < {n}; {v} += (long long)gridDim.x * blockDim.x) {{")
            shared = _shares(c.body) or self.sync[-1]
            self.sync.append(shared)
            self.emit(c.body, ind + 1, ctx + (c.level,))
            self.sync.pop()
            if (self.backend == "cuda" and shared and c.level in ("workgroup", "seq")
                    and _block_uniform(ctx) and _threaded(c.body)):
                # the next iteration's thread-level loops overwrite what this one's threads still read
                self.barrier(pad + "  ")
            self.lines.append(f"{pad}}}")
            return
        if isinstance(c, T.TreeReduce):
            self.emit_tree(c, ind, ctx)
            return
        if isinstance(c, T.LastBlock):
            self.emit_last_block(c, ind, ctx)
            return
        raise EmitError(f"unknown command {type(c).__name__}")

    def barrier(self, pad: str):
        """A block barrier, unless the line before is one already."""
        if not (self.lines and self.lines[-1].strip() == "__syncthreads();"):
            self.lines.append(f"{pad}__syncthreads();")

    def emit_tree(self, c: T.TreeReduce, ind: int, ctx: tuple):
        if isinstance(c.buf.type.elem, P.PairT):
            return self.emit_pair_tree(c, ind, ctx)
        pad = "  " * ind
        L = c.buf.type.n
        et = c.buf.type.elem
        bufv = P.Ident(c.buf.name, c.buf.type, temp="private")
        ct = ctype(et)
        zero = self.literal(P.Lit(0.0, et))
        self.private_ctx[c.buf.name] = (sum(1 for l in ctx if l != "seq"), _per_thread(ctx))
        if self.backend == "cuda":
            if "warp" not in ctx or "lane" in ctx:
                raise EmitError("a lane tree runs directly inside a warp loop")
            # lane l keeps element l; lanes past L hold zeros, which never reach lane 0
            self.lines.append(f"{pad}{ct} {c.buf.name} = {zero};")
            self.emit(c.fill, ind, ctx)
            reg = P.Ident(c.buf.name, et, temp="private")
            h = L // 2
            while h >= 1:  # every lane of the warp takes part in each shuffle
                step = P.apply(c.f, reg, Shuffle(reg, h))
                self.lines.append(f"{pad}{c.buf.name} = {self.access(step, [])};")
                h //= 2
            self.lines.append(f"{pad}{c.res.name} = {c.buf.name};  // the tree's value, in lane 0")
            return
        self.lines.append(f"{pad}{ct} {c.buf.name}[{L}];")
        self.emit(c.fill, ind, ctx)
        h = L // 2
        while h >= 1:
            j = T.IVar("dpia_l")
            step = P.apply(c.f, P.Idx(bufv, j), P.Idx(bufv, T.iadd(j, T.IConst(h))))
            self.lines.append(f"{pad}for (long long dpia_l = 0; dpia_l < {h}; ++dpia_l) "
                              f"{c.buf.name}[dpia_l] = {self.access(step, [])};")
            h //= 2
        self.lines.append(f"{pad}{c.res.name} = {c.buf.name}[0];")

    def emit_pair_tree(self, c: T.TreeReduce, ind: int, ctx: tuple):
        """The halving tree over pairs (e.g. compensated sums (s, c)): each step
        computes both components of f(x_l, x_{l+h}) before either replaces x_l
        (the second component may read the first's old value)."""
        pad = "  " * ind
        L = c.buf.type.n
        et = c.buf.type.elem
        ct = ctype(et.a)
        zero = self.literal(P.Lit(0.0, et.a))
        self.private_ctx[c.buf.name] = (sum(1 for l in ctx if l != "seq"), _per_thread(ctx))
        if isinstance(c.res.type, P.PairT):
            res = [f"{c.res.name}_0", f"{c.res.name}_1"]
        else:
            raise EmitError("a tree over pairs gives a pair")
        if self.backend == "cuda":
            if "warp" not in ctx or "lane" in ctx:
                raise EmitError("a lane tree runs directly inside a warp loop")
            # lane l keeps element l in two registers; lanes past L hold zeros
            self.lines.append(f"{pad}{ct} {c.buf.name}_0 = {zero};")
            self.lines.append(f"{pad}{ct} {c.buf.name}_1 = {zero};")
            self.emit(c.fill, ind, ctx)
            reg = P.Ident(c.buf.name, et, temp="private")
            other = P.Ident("dpia_o", et, temp="private")  # lane l + h's pair, shuffled once
            h = L // 2
            while h >= 1:
                step = P.apply(c.f, reg, other)
                a0, a1 = self.access(step, [("p", 0)]), self.access(step, [("p", 1)])
                self.lines.append(f"{pad}{{ const {ct} dpia_o_0 = __shfl_down_sync(0xffffffffu, {c.buf.name}_0, {h}); "
                                  f"const {ct} dpia_o_1 = __shfl_down_sync(0xffffffffu, {c.buf.name}_1, {h});")
                self.lines.append(f"{pad}  const {ct} dpia_n0 = {a0}; const {ct} dpia_n1 = {a1}; "
                                  f"{c.buf.name}_0 = dpia_n0; {c.buf.name}_1 = dpia_n1; }}")
                h //= 2
            self.lines.append(f"{pad}{res[0]} = {c.buf.name}_0;  // the tree's value, in lane 0")
            self.lines.append(f"{pad}{res[1]} = {c.buf.name}_1;")
            return
        bufv = P.Ident(c.buf.name, c.buf.type, temp="private")
        self.lines.append(f"{pad}{ct} {c.buf.name}[{2 * L}];")
        self.emit(c.fill, ind, ctx)
        h = L // 2
        while h >= 1:
            j = T.IVar("dpia_l")
            step = P.apply(c.f, P.Idx(bufv, j), P.Idx(bufv, T.iadd(j, T.IConst(h))))
            a0, a1 = self.access(step, [("p", 0)]), self.access(step, [("p", 1)])
            self.lines.append(f"{pad}for (long long dpia_l = 0; dpia_l < {h}; ++dpia_l) {{ "
                              f"const {ct} dpia_n0 = {a0}; const {ct} dpia_n1 = {a1}; "
                              f"{c.buf.name}[2 * dpia_l] = dpia_n0; {c.buf.name}[2 * dpia_l + 1] = dpia_n1; }}")
            h //= 2
        self.lines.append(f"{pad}{res[0]} = {c.buf.name}[0];")
        self.lines.append(f"{pad}{res[1]} = {c.buf.name}[1];")

    def emit_last_block(self, c: T.LastBlock, ind: int, ctx: tuple):
        pad = "  " * ind
        if ctx:
            raise EmitError("the second level runs outside every loop")
        inner = ("workgroup",)
        if self.backend == "c":
            self.emit(c.body, ind, inner)
            return
        tk = c.ticket.name
        self.shared.append("  __shared__ int dpia_last;")
        # the barrier orders every thread's writes of the parts before thread 0's
        # fence, whose release (cumulative) makes them visible before the ticket
        self.barrier(pad)
        self.lines += [f"{pad}if (threadIdx.x == 0) {{",
                       f"{pad}  __threadfence();",
                       f"{pad}  dpia_last = atomicAdd({tk}, 1) == (int)gridDim.x - 1;",
                       f"{pad}}}",
                       f"{pad}__syncthreads();",
                       f"{pad}if (dpia_last) {{",
                       f"{pad}  __threadfence();"]
        self.in_last = True
        self.sync.append(True)
        self.emit(c.body, ind + 1, inner)
        self.sync.pop()
        self.in_last = False
        self.lines += [f"{pad}  if (threadIdx.x == 0) {tk}[0] = 0;  // the counter is zero for the next launch",
                       f"{pad}}}"]

    def guard(self, ctx) -> str:
        if self.backend == "c" or "guarded" in ctx:
            return ""
        if "local" in ctx or "global" in ctx or "lane" in ctx:
            return ""
        if "warp" in ctx:
            return "if ((threadIdx.x & 31) == 0) "
        if "workgroup" in ctx:
            return "if (threadIdx.x == 0) "
        return "if (blockIdx.x == 0 && threadIdx.x == 0) "

    @staticmethod
    def has_parallel(c) -> bool:
        if isinstance(c, T.For):
            return c.level != "seq" or Emitter.has_parallel(c.body)
        if isinstance(c, T.Seq):
            return any(Emitter.has_parallel(x) for x in c.cs)
        if isinstance(c, T.New):
            return Emitter.has_parallel(c.body)
        if isinstance(c, (T.TreeReduce, T.LastBlock)):
            return True
        return False

    def check_private_reads(self, e, ctx):
        """A private value is visible to its own thread only: one declared where
        a single thread computes it may not be read inside a thread-level loop."""
        if self.backend != "cuda":
            return
        inside_threads = _per_thread(ctx)
        for name in _idents(e):
            if name in self.private_ctx:
                _, declared_inside = self.private_ctx[name]
                if inside_threads and not declared_inside:
                    raise EmitError(f"private value {name} is computed by one thread but read by "
                                    f"all threads of a thread-level map; place it in local memory")


def _shared_bytes(decl: str) -> int:
    """Bytes of a '__shared__ T name[count];' (or scalar 'T name;') declaration, 4-byte elements."""
    return 4 * int(decl.split("[")[1].split("]")[0]) if "[" in decl else 4


class Shuffle(P.Phrase):
    """The value of e in the lane ``offset`` lanes above this one (emitted by
    the lane tree only)."""

    def __init__(self, e, offset: int):
        self.e, self.offset, self.type = e, offset, e.type

    def children(self):
        return (self.e,)


def _block_uniform(ctx) -> bool:
    """Every thread of the block runs code in ctx (no thread-level loop or guard
    around it), so a block barrier there is reached by all of them."""
    return not (set(ctx) & {"local", "global", "warp", "lane", "guarded"})


def _per_thread(ctx) -> bool:
    """Code in ctx runs once per thread (inside a local, global or lane loop)."""
    return "local" in ctx or "global" in ctx or "lane" in ctx


def _shares(c) -> bool:
    """c declares a temporary in local or global memory."""
    if isinstance(c, T.New):
        return c.temp.space != "private" or _shares(c.body)
    if isinstance(c, T.For):
        return _shares(c.body)
    if isinstance(c, T.Seq):
        return any(_shares(x) for x in c.cs)
    if isinstance(c, T.TreeReduce):
        return _shares(c.fill)
    return False


def _has_level(c, level) -> bool:
    if isinstance(c, T.For):
        return c.level == level or _has_level(c.body, level)
    if isinstance(c, T.Seq):
        return any(_has_level(x, level) for x in c.cs)
    if isinstance(c, T.New):
        return _has_level(c.body, level)
    if isinstance(c, T.TreeReduce):
        return c.level == level or _has_level(c.fill, level)
    if isinstance(c, T.LastBlock):
        return _has_level(c.body, level)
    return False


def _threaded(c) -> bool:
    """c runs loops spread over the block's threads (its reads and writes of
    shared temporaries need barriers around them)."""
    return any(_has_level(c, lvl) for lvl in THREADED)


def _idents(e):
    if isinstance(e, P.Ident):
        yield e.name
    for c in e.children():
        yield from _idents(c)


def generate(name: str, expr: P.Phrase, inputs: list, backend: str = "cuda", unroll: int = 1) -> dict:
    """Source of a kernel computing expr into an output array; ``unroll`` > 1
    asks the CUDA compiler to unroll sequential loops by that factor.

    Returns {"source", "kernel", "params" (name, C type, count, role), "temps"}.
    """
    import re

    for p in inputs:
        if not re.fullmatch(r"[A-Za-z_][A-Za-z_0-9]*", p.name) or re.fullmatch(r"[tirl]\d+|out|dpia_\w*", p.name):
            raise EmitError(f"input name {p.name!r}: a C identifier other than out, dpia_*, t<k>, i<k>, r<k>, "
                            f"l<k>")
    if len({p.name for p in inputs}) != len(inputs):
        raise EmitError("two inputs share a name")
    comm, out = T.translate(expr, "out")
    temps = T.hoist(comm)
    from .check import check
    from .typecheck import typecheck

    typecheck(comm, out)  # phrase types, passive parallel bodies, legal nesting (race-free by construction)
    check(comm)  # and, on the index arithmetic: no two iterations of a parallel loop write one place
    em = Emitter(backend, inputs, out, temps, unroll)
    em.emit(comm, 1, ())
    params = []
    for p in inputs:
        ct = CTYPE[P.base_num(p.type).dtype]
        params.append((p.name, ct, P.scalar_count(p.type) if isinstance(p.type, P.Arr) else 1, "in"))
    params.append(("out", CTYPE[P.base_num(expr.type).dtype],
                   P.scalar_count(expr.type) if isinstance(expr.type, P.Arr) else 1, "out"))
    for t in temps:
        if t.space == "global":
            count = P.scalar_count(t.type)
            for _, n in t.hoist:
                count *= n
            params.append((t.name, CTYPE[P.base_num(t.type).dtype], count, "temp"))
    sig = []
    for pname, ct, _, role in params:
        if role == "in":
            sig.append(f"const {ct} *__restrict__ {pname}")
        else:
            sig.append(f"{ct} *__restrict__ {pname}")
    body = "\n".join(em.shared + em.lines)
    if backend == "cuda":
        src = (f"{CUDA_PRELUDE}\nextern \"C\" __global__ void {name}({', '.join(sig)}) {{\n{body}\n}}\n")
    else:
        src = f"{C_PRELUDE}\nvoid {name}({', '.join(sig)}) {{\n{body}\n}}\n"
    return {"source": src, "kernel": name, "params": params, "temps": temps, "comm": comm}
