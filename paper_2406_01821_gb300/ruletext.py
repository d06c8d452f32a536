"""Readable and tensor forms of rule sets (the layouts of the paper's Fig. 1).

* Readable form (Fig. 1b / 1c): one line per rule,
  ``1. (mean radius > 2.02) & (fractal dimension error > 0.38 x worst compactness) -> malignant``,
  plus, in this library's format, a final ``else -> <class>`` line for the default class.
  A condition is ``(lhs op rhs)`` with op ``>`` or ``<``; ``lhs`` is ``name`` (a = 1), ``-name``
  (a = -1) or ``a x name``; ``rhs`` is a threshold ``t`` or ``b x name``. A membership test on a
  categorical feature reads ``(name in {0, 2, 5})`` (its category codes).
* Tensor form (Fig. 1a): one row per condition, ``sum_j w_j x_j + bias > 0``. A threshold
  condition ``a x_f > t`` is the row w_f = a, bias = -t; a feature pair ``a x_f > b x_g`` is
  w_f = a, w_g = -b, bias 0. A ``<`` condition is written as the row of the negated ``>`` form
  (the figure has only ``>`` rows; the negation is exact in float32).

``render`` with ``digits=None`` prints every number as the shortest decimal that reads back to
the same float32, so ``parse(render(...))`` reproduces the batch bit for bit; ``digits=2`` gives
the two-decimal display of the figure.
"""
from __future__ import annotations

from typing import List, Optional, Sequence, Tuple

import numpy as np

from . import synth

Cond = tuple                                          # (f, g, op, a, b, t[, codes]), g = -1: threshold
Rule = Tuple[int, List[Cond]]                          # (class, conditions)


def _num(v: float, digits: Optional[int]) -> str:
    v = np.float32(v)
    if np.isnan(v):
        return "nan"
    if np.isinf(v):
        return "inf" if v > 0 else "-inf"
    if digits is not None:
        return f"{float(v):.{digits}f}"
    return np.format_float_positional(v, unique=True, trim="-") if abs(v) >= 1e-4 or v == 0 \
        else np.format_float_scientific(v, unique=True, trim="-")


def _term(coef: float, name: str, digits: Optional[int]) -> str:
    c = np.float32(coef)
    if c == 1.0 and not np.signbit(c):
        return name
    if c == -1.0:
        return "-" + name
    return f"{_num(c, digits)} x {name}"


def set_rules(batch: synth.Batch, p: int) -> Tuple[List[Rule], int]:
    """Rules of set p as (class, [(f, g, op, a, b, t), ...]) and its default class; a membership
    condition carries its category codes as a seventh element."""
    rules = []
    for r in range(batch.set_rule_off[p], batch.set_rule_off[p + 1]):
        conds = []
        for c in range(batch.rule_cond_off[r], batch.rule_cond_off[r + 1]):
            cond = (int(batch.cond_f[c]), int(batch.cond_g[c]), int(batch.cond_op[c]),
                    float(batch.cond_a[c]), float(batch.cond_b[c]), float(batch.cond_t[c]))
            if cond[2] == synth.IN:
                cond += (synth.category_codes(int(batch.cond_set[c])),)
            conds.append(cond)
        rules.append((int(batch.rule_class[r]), conds))
    return rules, int(batch.set_default[p])


def render_rules(rules: Sequence[Rule], features: Sequence[str], classes: Sequence[str],
                 default: Optional[int] = None, digits: Optional[int] = None) -> List[str]:
    """Readable lines of one rule set (Fig. 1b layout); ``default`` adds the ``else`` line."""
    out = []
    for i, (cls, conds) in enumerate(rules):
        parts = []
        for cond in conds:
            f, g, op, a, b, t = cond[:6]
            if op == synth.IN:
                parts.append(f"({features[f]} in {{" + ", ".join(str(k) for k in cond[6]) + "})")
                continue
            sym = ">" if op == synth.GT else "<"
            rhs = _num(t, digits) if g < 0 else _term(b, features[g], digits)
            parts.append(f"({_term(a, features[f], digits)} {sym} {rhs})")
        out.append(f"{i + 1}. " + " & ".join(parts) + f" -> {classes[cls]}")
    if default is not None:
        out.append(f"else -> {classes[default]}")
    return out


def render(batch: synth.Batch, p: int, features: Optional[Sequence[str]] = None,
           classes: Optional[Sequence[str]] = None, digits: Optional[int] = None) -> List[str]:
    """Readable lines of set p of a batch, default class included."""
    rules, default = set_rules(batch, p)
    nf = 1 + max([max(cd[0], cd[1]) for _, cs in rules for cd in cs], default=0)
    nk = 1 + max([cls for cls, _ in rules] + [default])
    features = features or [f"x{j}" for j in range(nf)]
    classes = classes or [f"class{k}" for k in range(nk)]
    return render_rules(rules, features, classes, default, digits)


def _parse_term(s: str, features: Sequence[str]) -> Tuple[float, int]:
    s = s.strip()
    if " x " in s:
        c, name = s.split(" x ", 1)
        return float(np.float32(c)), list(features).index(name)
    if s.startswith("-") and s[1:] in features:
        return -1.0, list(features).index(s[1:])
    return 1.0, list(features).index(s)


def parse_rules(lines: Sequence[str], features: Sequence[str],
                classes: Sequence[str]) -> Tuple[List[Rule], Optional[int]]:
    """Inverse of ``render_rules``: rules and the default class (None without an ``else`` line)."""
    rules, default = [], None
    for ln in lines:
        ln = ln.strip()
        if not ln:
            continue
        body, cls = ln.rsplit(" -> ", 1)
        k = list(classes).index(cls.strip())
        if body.strip() == "else":
            default = k
            continue
        body = body.split(". ", 1)[1]
        conds: List[Cond] = []
        for part in _split_conditions(body):
            part = part.strip()[1:-1]
            if " in {" in part:
                name, codes = part.split(" in {", 1)
                ks = [int(v) for v in codes.rstrip("}").split(",") if v.strip()]
                conds.append((list(features).index(name.strip()), -1, synth.IN, 0.0, 0.0, 0.0, ks))
                continue
            op = synth.GT if " > " in part else synth.LT
            lhs, rhs = part.split(" > " if op == synth.GT else " < ")
            a, f = _parse_term(lhs, features)
            try:
                t = float(np.float32(rhs))
                conds.append((f, -1, op, a, 0.0, t))
            except ValueError:
                b, g = _parse_term(rhs, features)
                conds.append((f, g, op, a, b, 0.0))
        rules.append((k, conds))
    return rules, default


def _split_conditions(body: str) -> List[str]:
    """The parenthesised conditions of a rule body, split at the top-level ' & '."""
    out, depth, start = [], 0, 0
    for i, ch in enumerate(body):
        depth += ch == "("
        depth -= ch == ")"
        if depth == 0 and body.startswith(" & ", i):
            out.append(body[start:i])
            start = i + 3
    out.append(body[start:])
    return out


def parse(texts: Sequence[Sequence[str]], features: Sequence[str], classes: Sequence[str],
          default: int = 0) -> synth.Batch:
    """A batch from the readable form of several rule sets (``default`` where a set has no
    ``else`` line)."""
    sets, defaults = [], []
    for lines in texts:
        rules, d = parse_rules(lines, features, classes)
        sets.append(rules)
        defaults.append(default if d is None else d)
    return synth.from_lists(sets, defaults)


def tensor_rows(rules: Sequence[Rule], F: int) -> List[Tuple[int, np.ndarray, float]]:
    """Fig. 1a rows: (class of the rule, weights [F], bias) per condition, in rule order.

    A pair whose coefficient b is 0 reads back as the threshold a*x_f > 0 (the two differ only
    where x_g is NaN); a pair on one feature and a zero threshold coefficient have no row."""
    rows = []
    for cls, conds in rules:
        for cond in conds:
            f, g, op, a, b, t = cond[:6]
            if op == synth.IN:
                raise ValueError("a membership test has no row form")
            if g == f or (g < 0 and a == 0.0):
                raise ValueError("a pair on one feature or a zero threshold coefficient has no row form")
            w = np.zeros(F, np.float32)
            s = np.float32(1.0 if op == synth.GT else -1.0)
            if g < 0:
                w[f] = s * np.float32(a)
                bias = -s * np.float32(t)
            else:
                w[f] += s * np.float32(a)
                w[g] += -s * np.float32(b)
                bias = np.float32(0.0)
            rows.append((cls, w, float(bias)))
    return rows


def from_tensor_rows(rows: Sequence[Tuple[int, Sequence[float], float]],
                     rule_sizes: Sequence[int]) -> List[Rule]:
    """Rules from Fig. 1a rows: one non-zero weight w_f with bias beta is a*x_f > t with a = w_f,
    t = -beta; two non-zeros w_f, w_g (bias 0) are a*x_f > b*x_g with a = w_f, b = -w_g."""
    rules: List[Rule] = []
    it = iter(rows)
    for size in rule_sizes:
        conds: List[Cond] = []
        cls = None
        for _ in range(size):
            cls, w, bias = next(it)
            nz = [j for j, v in enumerate(w) if v != 0.0]
            if len(nz) == 1:
                f = nz[0]
                conds.append((f, -1, synth.GT, float(w[f]), 0.0, float(-np.float32(bias))))
            elif len(nz) == 2 and bias == 0.0:
                f, g = nz
                conds.append((f, g, synth.GT, float(w[f]), float(-np.float32(w[g])), 0.0))
            else:
                raise ValueError("a row has one non-zero weight, or two and a zero bias")
        rules.append((int(cls) if cls is not None else 0, conds))
    return rules
