"""Parse and normalise association trees for the golden-tree pins.

Grammar of the golden expressions: sum := prod ('+' prod)* (left associative),
prod := atom ('*' atom)*, atom := '(' sum ')' | '|' name '|' | name | '0'.
Normal form: products with a literal 0 factor become 0, additions of 0 are
dropped, and the operands of + and * are sorted (both commute exactly in IEEE
arithmetic), so two trees are equal iff they add the same products in the same
bracketing.
"""
from __future__ import annotations

import re

_TOK = re.compile(r"\s*(\(|\)|\+|\*|\||[A-Za-z_][A-Za-z_0-9]*|0)")


def parse(text: str):
    toks = _TOK.findall(text)
    if "".join(toks) != re.sub(r"\s+", "", text):
        raise ValueError(f"bad expression: {text}")
    pos = 0

    def peek():
        return toks[pos] if pos < len(toks) else None

    def take(t=None):
        nonlocal pos
        tok = toks[pos]
        if t is not None and tok != t:
            raise ValueError(f"expected {t} got {tok}")
        pos += 1
        return tok

    def atom():
        t = peek()
        if t == "(":
            take("(")
            e = sum_()
            take(")")
            return e
        if t == "|":
            take("|")
            name = take()
            take("|")
            return ("abs", name)
        return take()

    def prod():
        e = atom()
        while peek() == "*":
            take("*")
            e = ("*", e, atom())
        return e

    def sum_():
        e = prod()
        while peek() == "+":
            take("+")
            e = ("+", e, prod())
        return e

    e = sum_()
    if pos != len(toks):
        raise ValueError(f"trailing tokens in {text}")
    return e


def _key(t):
    return repr(t)


def normalise(t):
    if isinstance(t, str):
        return t
    op = t[0]
    if op == "abs":
        return ("abs", normalise(t[1]))
    a, b = normalise(t[1]), normalise(t[2])
    if op == "*":
        if a == "0" or b == "0":
            return "0"
    if op == "+":
        if a == "0":
            return b
        if b == "0":
            return a
    if op in ("+", "*"):
        a, b = sorted((a, b), key=_key)
    return (op, a, b)


def symbols(n, prefix):
    return [f"{prefix}{i}" for i in range(n)]


def load_golden(path):
    entries, cur = [], {}
    with open(path) as f:
        for line in f:
            line = line.rstrip("\n")
            if not line.strip() or line.lstrip().startswith("#"):
                if cur:
                    entries.append(cur)
                    cur = {}
                continue
            k, _, v = line.partition(":")
            cur[k.strip()] = v.strip()
    if cur:
        entries.append(cur)
    return entries


def strategy_fields(text):
    out = {}
    for part in text.split():
        k, _, v = part.partition("=")
        out[k] = v
    return out
