"""OpenQASM 2.0 front end: circuits as text -> gate lists of ``inputs``.

The paper runs circuits given in OpenQASM (Sec. II: the simulator takes
OpenQASM and other front ends).  This parser covers the part of the language
a gate-level simulator needs:

* ``OPENQASM 2.0;``, ``include "...";`` (the standard gate names below are
  built in, nothing is read from disk), ``qreg`` (several registers are laid
  out one after the other: the first register's qubit 0 is qubit 0),
  ``creg``, ``barrier`` and ``measure`` (no effect on the state; the
  measured qubits are recorded);
* gate applications with register broadcasting (``h q;``, ``cx a, b;`` on
  equal-size registers);
* parameter expressions: numbers, ``pi``, + - * / ^, unary minus,
  parentheses and sin, cos, tan, exp, ln, sqrt;
* user ``gate`` definitions, expanded at each use.

Built-in gates: id/u0, x, y, z, h, s, sdg, t, tdg, sx, rx, ry, rz, p/u1,
u2, u3/u/U, cx/CX, cz, swap, rzz, and the controlled gates cp/cu1, crz,
cy, ch as 4x4 matrices (first argument = control).  ``rz`` is the rotation
exp(-i theta Z / 2), ``p``/``u1`` the phase gate diag(1, e^{i lambda})
(they differ by a global phase, which no observable sees).  ``reset``,
``if`` and ``opaque`` are rejected, as are gates on three or more qubits
unless the program defines them.
"""
from __future__ import annotations

import math
import re

import numpy as np

from . import inputs

_SIMPLE = {"id": "ID", "u0": "ID", "x": "X", "y": "Y", "z": "Z", "h": "H", "s": "S", "sdg": "SDG", "t": "T",
           "tdg": "TDG", "sx": "SX"}
_ROT = {"rx": "RX", "ry": "RY", "rz": "RZ", "p": "P", "u1": "P"}
_TWO = {"cx": "CX", "CX": "CX", "cz": "CZ", "swap": "SWAP"}
_NPARAM = {"rx": 1, "ry": 1, "rz": 1, "p": 1, "u1": 1, "u2": 2, "u3": 3, "u": 3, "U": 3, "rzz": 1, "cp": 1,
           "cu1": 1, "crz": 1}
_FUNCS = {"sin": math.sin, "cos": math.cos, "tan": math.tan, "exp": math.exp, "ln": math.log, "sqrt": math.sqrt}


class QasmError(ValueError):
    pass


# ---------------------------------------------------------------- expressions
_TOK = re.compile(r"\s*(?:(\d+\.\d*(?:[eE][-+]?\d+)?|\.\d+(?:[eE][-+]?\d+)?|\d+(?:[eE][-+]?\d+)?)|([A-Za-z_]\w*)|(.))")


def _tokens(s):
    pos, out = 0, []
    s = s.strip()
    while pos < len(s):
        m = _TOK.match(s, pos)
        if not m or m.end() == pos:
            raise QasmError(f"bad expression {s!r}")
        num, name, op = m.groups()
        if num is not None:
            out.append(("num", float(num)))
        elif name is not None:
            out.append(("name", name))
        elif op.strip():
            out.append(("op", op))
        pos = m.end()
    return out


def evaluate(expr, env=None):
    """Value of a parameter expression; ``env`` maps parameter names to values."""
    env = env or {}
    toks = _tokens(expr)
    i = 0

    def peek():
        return toks[i] if i < len(toks) else (None, None)

    def take(kind=None, val=None):
        nonlocal i
        t = peek()
        if t[0] is None or (kind and t[0] != kind) or (val and t[1] != val):
            raise QasmError(f"bad expression {expr!r}")
        i += 1
        return t

    def atom():
        k, v = peek()
        if k == "num":
            take()
            return v
        if k == "name":
            take()
            if v == "pi":
                return math.pi
            if v in _FUNCS:
                take("op", "(")
                x = add()
                take("op", ")")
                return _FUNCS[v](x)
            if v in env:
                return env[v]
            raise QasmError(f"unknown name {v!r} in expression")
        if (k, v) == ("op", "("):
            take()
            x = add()
            take("op", ")")
            return x
        if (k, v) == ("op", "-"):
            take()
            return -power()
        if (k, v) == ("op", "+"):
            take()
            return power()
        raise QasmError(f"bad expression {expr!r}")

    def power():
        x = atom()
        if peek() == ("op", "^"):
            take()
            return x ** power()  # right associative
        return x

    def mul():
        x = power()
        while peek() in (("op", "*"), ("op", "/")):
            op = take()[1]
            y = power()
            x = x * y if op == "*" else x / y
        return x

    def add():
        x = mul()
        while peek() in (("op", "+"), ("op", "-")):
            op = take()[1]
            y = mul()
            x = x + y if op == "+" else x - y
        return x

    v = add()
    if i != len(toks):
        raise QasmError(f"bad expression {expr!r}")
    return float(v)


def _split_args(s):
    """Split at top-level commas."""
    out, depth, cur = [], 0, ""
    for ch in s:
        if ch == "," and depth == 0:
            out.append(cur)
            cur = ""
            continue
        depth += ch == "("
        depth -= ch == ")"
        cur += ch
    if cur.strip():
        out.append(cur)
    return [a.strip() for a in out]


# ---------------------------------------------------------------- built-in gates
def _builtin(name, params, qubits):
    """Gate tuples of one built-in application (qubits already resolved)."""
    if name in _SIMPLE:
        return [inputs.gate(_SIMPLE[name], qubits)]
    if name in _ROT:
        return [inputs.gate(_ROT[name], qubits, params)]
    if name == "u2":
        return [inputs.gate("U3", qubits, (math.pi / 2, params[0], params[1]))]
    if name in ("u3", "u", "U"):
        return [inputs.gate("U3", qubits, params)]
    if name in _TWO:
        return [inputs.gate(_TWO[name], qubits)]
    if name == "rzz":
        return [inputs.gate("RZZ", qubits, params)]
    if name in ("cp", "cu1", "crz", "cy", "ch"):
        if name in ("cp", "cu1"):
            U = np.diag([1.0, np.exp(1j * params[0])])
        elif name == "crz":
            U = np.diag([np.exp(-0.5j * params[0]), np.exp(0.5j * params[0])])
        elif name == "cy":
            U = np.array([[0, -1j], [1j, 0]])
        else:
            U = np.array([[1, 1], [1, -1]]) / math.sqrt(2.0)
        M = np.eye(4, dtype=complex)
        M[np.ix_([1, 3], [1, 3])] = U
        return [inputs.gate("MAT2", qubits, M)]
    raise QasmError(f"unknown gate {name!r}")


_BUILTIN_ARITY = {**{k: 1 for k in list(_SIMPLE) + list(_ROT) + ["u2", "u3", "u", "U"]},
                  **{k: 2 for k in list(_TWO) + ["rzz", "cp", "cu1", "crz", "cy", "ch"]}}


# ---------------------------------------------------------------- parser
_STMT_GATE = re.compile(r"^([A-Za-z_]\w*)\s*(?:\((.*)\))?\s+(.+)$", re.S)


class _Program:
    def __init__(self):
        self.regs = {}  # name -> (offset, size)
        self.n = 0
        self.defs = {}  # name -> (param names, arg names, body statements)
        self.gates = []
        self.measured = []

    def resolve(self, arg):
        """'q[3]' -> [qubit], 'q' -> all qubits of q."""
        m = re.fullmatch(r"([A-Za-z_]\w*)\s*(?:\[\s*(\d+)\s*\])?", arg)
        if not m or m.group(1) not in self.regs:
            raise QasmError(f"unknown register operand {arg!r}")
        off, size = self.regs[m.group(1)]
        if m.group(2) is None:
            return [off + i for i in range(size)]
        i = int(m.group(2))
        if i >= size:
            raise QasmError(f"index out of range in {arg!r}")
        return [off + i]

    def apply(self, name, params, qubits, depth=0):
        if depth > 64:
            raise QasmError("gate definitions nest too deeply")
        if name in self.defs:
            pnames, anames, body = self.defs[name]
            if len(params) != len(pnames) or len(qubits) != len(anames):
                raise QasmError(f"wrong parameter or argument count for {name!r}")
            env = dict(zip(pnames, params))
            amap = dict(zip(anames, qubits))
            for st in body:
                m = _STMT_GATE.match(st)
                if not m:
                    raise QasmError(f"bad statement in gate {name!r}: {st!r}")
                sub, pe, ae = m.group(1), m.group(2), m.group(3)
                if sub == "barrier":
                    continue
                sp = [evaluate(x, env) for x in _split_args(pe)] if pe else []
                try:
                    sq = [amap[a] for a in _split_args(ae)]
                except KeyError as e:
                    raise QasmError(f"unknown argument {e} in gate {name!r}") from None
                self.apply(sub, sp, sq, depth + 1)
            return
        if name not in _BUILTIN_ARITY:
            raise QasmError(f"unknown gate {name!r}")
        if len(qubits) != _BUILTIN_ARITY[name] or len(params) != _NPARAM.get(name, 0):
            raise QasmError(f"wrong parameter or argument count for {name!r}")
        if len(set(qubits)) != len(qubits):
            raise QasmError(f"repeated qubit in {name!r}")
        self.gates += _builtin(name, params, tuple(qubits))

    def statement(self, st):
        st = st.strip()
        if not st:
            return
        head = st.split(None, 1)[0]
        if head == "OPENQASM":
            if not re.fullmatch(r"OPENQASM\s+2(\.0)?", st):
                raise QasmError("only OpenQASM 2.0 is supported")
            return
        if head == "include":
            return
        m = re.fullmatch(r"(qreg|creg)\s+([A-Za-z_]\w*)\s*\[\s*(\d+)\s*\]", st)
        if m:
            if m.group(1) == "qreg":
                size = int(m.group(3))
                self.regs[m.group(2)] = (self.n, size)
                self.n += size
            return
        m = re.match(r"(reset|if|opaque)\b", st)
        if m:
            raise QasmError(f"{m.group(1)!r} is not supported")
        if head == "barrier":
            return
        if head == "measure":
            m = re.fullmatch(r"measure\s+(.+?)\s*->\s*(.+)", st)
            if not m:
                raise QasmError(f"bad measure statement {st!r}")
            self.measured += self.resolve(m.group(1))
            return
        m = _STMT_GATE.match(st)
        if not m:
            raise QasmError(f"bad statement {st!r}")
        name, pe, ae = m.group(1), m.group(2), m.group(3)
        params = [evaluate(x) for x in _split_args(pe)] if pe else []
        operands = [self.resolve(a) for a in _split_args(ae)]
        width = max(len(o) for o in operands)
        if any(len(o) not in (1, width) for o in operands):
            raise QasmError(f"registers of different sizes in {st!r}")
        for i in range(width):  # broadcasting over whole registers
            self.apply(name, params, [o[i] if len(o) > 1 else o[0] for o in operands])


def parse(text):
    """Parse an OpenQASM 2.0 program.  Returns dict(n=qubits, gates=[gate
    tuples], measured=[qubits in measure statements])."""
    text = re.sub(r"//[^\n]*", "", text)
    prog = _Program()
    pos = 0
    while True:
        m = re.search(r"\bgate\s+([A-Za-z_]\w*)\s*(?:\(([^)]*)\))?\s*([^{]*)\{([^}]*)\}", text[pos:])
        # statements before the next gate definition
        end = pos + (m.start() if m else len(text) - pos)
        for st in text[pos:end].split(";"):
            prog.statement(st)
        if not m:
            break
        name = m.group(1)
        pnames = [p.strip() for p in m.group(2).split(",")] if m.group(2) and m.group(2).strip() else []
        anames = [a.strip() for a in m.group(3).split(",") if a.strip()]
        body = [s.strip() for s in m.group(4).split(";") if s.strip()]
        prog.defs[name] = (pnames, anames, body)
        pos = pos + m.end()
    if prog.n == 0:
        raise QasmError("no qreg declared")
    return dict(n=prog.n, gates=prog.gates, measured=prog.measured)


def dumps(n, gates):
    """OpenQASM 2.0 text of a gate list (MAT1/MAT2 are not expressible)."""
    names = {"ID": "id", "X": "x", "Y": "y", "Z": "z", "H": "h", "S": "s", "SDG": "sdg", "T": "t", "TDG": "tdg",
             "SX": "sx", "RX": "rx", "RY": "ry", "RZ": "rz", "P": "p", "U3": "u3", "CX": "cx", "CZ": "cz",
             "SWAP": "swap", "RZZ": "rzz"}
    lines = ["OPENQASM 2.0;", 'include "qelib1.inc";', f"qreg q[{n}];"]
    for name, qs, prm in gates:
        if name not in names:
            raise QasmError(f"{name} has no OpenQASM form")
        p = "(" + ",".join(repr(float(x)) for x in prm) + ")" if prm else ""
        lines.append(f"{names[name]}{p} " + ",".join(f"q[{q}]" for q in qs) + ";")
    return "\n".join(lines) + "\n"
