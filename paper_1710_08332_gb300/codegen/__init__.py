"""A strategy-preserving code generator: functional phrases over the paper's
primitives (map at a level of the hierarchy -- work-group, warp, lane,
local, sequential --, reduceSeq, zip, split, join, transpose, address-space
annotations, lane trees and the last work-group's second level) are translated to an imperative loop
nest (acceptor- and continuation-passing translations, then the mapI /
reduceI expansion) and emitted as CUDA C for sm_103a or as C for the host.
The emitted code evaluates exactly the tree the phrase denotes, so its
results are bit-identical to any other evaluation of the same phrase.
"""
from .build import CFunction, CudaKernel, compile_c, compile_cuda
from .emit import EmitError, generate
from .phrase import (F32, I32, I64, Arr, Num, PairT, VecT, abs_, add, alit, arr, fma, asScalar, asVector, fst, inp, join,
                     lanes, lit, mapGlobal, mapLane, mapLocal, mapSeq, mapWarp, mapWorkgroup, mul, reduceSeq,
                     reduceTree, secondLevel, snd, splat, split, sub, to_global, to_local, to_private, transpose, vlit, zip_)
from .translate import TranslationError
from .typecheck import TypeCheckError

__all__ = [n for n in dir() if not n.startswith("_")]
