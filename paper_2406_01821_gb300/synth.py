"""Seeded synthetic workloads: tabular datasets and populations of ordered rule sets.

This module only draws random inputs. It holds none of the evaluation arithmetic: the CPU
oracle and the CUDA path both receive the arrays built here and nothing else.

Shapes and value laws follow the workloads of the paper's experiments (Sec. 4.1: a tabular
two-class dataset of 569 samples x 30 features, a pool of candidate rule sets) scaled up to the
batch sizes the library is built for. The UCI Breast Cancer records themselves are not used or
reproduced; a Gaussian two-class generator of the same shape stands in for them.

Rule-set batch layout (the C-ABI ``rs_batch`` layout, all arrays contiguous):
  set_rule_off  int32[P+1]   rules of set p are [set_rule_off[p], set_rule_off[p+1])
  rule_cond_off int32[R+1]   conditions of rule r are [rule_cond_off[r], rule_cond_off[r+1])
  rule_class    int32[R]     class named by rule r
  set_default   int32[P]     class assigned when no rule of set p fires
  cond_f, cond_g int32[C]    feature indices; cond_g = -1 marks a threshold condition
  cond_op       int8[C]      0: '>' , 1: '<', 2: category membership
  cond_a, cond_b, cond_t float32[C]
  cond_set      uint64[C] or None   category sets of membership conditions (bit k: code k)
A threshold condition reads  a*x[f] op t ; a feature-pair condition reads  a*x[f] op b*x[g]
(Sec. 3, Fig. 1a/1b). A membership condition (categorical features, named as future work in
Sec. 5) reads  x[f] in S : x[f] is an integer code k in 0..63 with bit k of cond_set set.
"""
from __future__ import annotations

import dataclasses
import numpy as np

GT, LT, IN = 0, 1, 2


@dataclasses.dataclass
class Batch:
    set_rule_off: np.ndarray
    rule_cond_off: np.ndarray
    rule_class: np.ndarray
    set_default: np.ndarray
    cond_f: np.ndarray
    cond_g: np.ndarray
    cond_op: np.ndarray
    cond_a: np.ndarray
    cond_b: np.ndarray
    cond_t: np.ndarray
    cond_set: np.ndarray | None = None

    @property
    def P(self) -> int:
        return int(self.set_default.shape[0])

    @property
    def R(self) -> int:
        return int(self.rule_class.shape[0])

    @property
    def C(self) -> int:
        return int(self.cond_f.shape[0])

    def nominal_conditions(self) -> int:
        """Sum over sets and rules of the rule's condition count."""
        return int(self.rule_cond_off[-1])

    def arrays(self):
        return {f.name: getattr(self, f.name) for f in dataclasses.fields(self)
                if getattr(self, f.name) is not None}

    def nbytes(self) -> int:
        return sum(a.nbytes for a in self.arrays().values())

    def subset(self, sets) -> "Batch":
        """A batch holding only the listed sets (in the given order)."""
        sets = np.asarray(sets, dtype=np.int64)
        rule_lists = [np.arange(self.set_rule_off[p], self.set_rule_off[p + 1]) for p in sets]
        rules = np.concatenate(rule_lists) if rule_lists else np.zeros(0, np.int64)
        set_rule_off = np.zeros(len(sets) + 1, np.int32)
        set_rule_off[1:] = np.cumsum([len(r) for r in rule_lists])
        cond_lists = [np.arange(self.rule_cond_off[r], self.rule_cond_off[r + 1]) for r in rules]
        conds = np.concatenate(cond_lists) if cond_lists else np.zeros(0, np.int64)
        rule_cond_off = np.zeros(len(rules) + 1, np.int32)
        rule_cond_off[1:] = np.cumsum([len(c) for c in cond_lists])
        return Batch(set_rule_off, rule_cond_off,
                     self.rule_class[rules].astype(np.int32), self.set_default[sets].astype(np.int32),
                     self.cond_f[conds].astype(np.int32), self.cond_g[conds].astype(np.int32),
                     self.cond_op[conds].astype(np.int8), self.cond_a[conds].astype(np.float32),
                     self.cond_b[conds].astype(np.float32), self.cond_t[conds].astype(np.float32),
                     None if self.cond_set is None else self.cond_set[conds].astype(np.uint64))


def from_lists(sets, defaults) -> Batch:
    """Build a batch from nested python lists.

    ``sets[p]`` is a list of rules; a rule is ``(cls, [cond, ...])`` and a condition is
    ``(f, g, op, a, b, t)`` with ``g = -1`` for a threshold condition, or
    ``(f, -1, IN, 0, 0, 0, codes)`` for a membership condition on the category codes ``codes``.
    The batch carries ``cond_set`` only when some condition is a membership test.
    """
    set_rule_off = [0]
    rule_cond_off = [0]
    rule_class, cf, cg, cop, ca, cb, ct, cs = [], [], [], [], [], [], [], []
    for rules in sets:
        for cls, conds in rules:
            rule_class.append(cls)
            for cond in conds:
                f, g, op, a, b, t = cond[:6]
                cf.append(f); cg.append(g); cop.append(op); ca.append(a); cb.append(b); ct.append(t)
                cs.append(category_mask(cond[6]) if len(cond) > 6 else 0)
            rule_cond_off.append(len(cf))
        set_rule_off.append(len(rule_class))
    return Batch(np.array(set_rule_off, np.int32), np.array(rule_cond_off, np.int32),
                 np.array(rule_class, np.int32), np.array(defaults, np.int32),
                 np.array(cf, np.int32), np.array(cg, np.int32), np.array(cop, np.int8),
                 np.array(ca, np.float32), np.array(cb, np.float32), np.array(ct, np.float32),
                 np.array(cs, np.uint64) if any(op == IN for op in cop) else None)


def category_mask(codes) -> int:
    """64-bit set of category codes (each 0..63)."""
    m = 0
    for k in codes:
        if not 0 <= int(k) <= 63:
            raise ValueError("category codes are 0..63")
        m |= 1 << int(k)
    return m


def category_codes(mask: int):
    """Sorted codes of a 64-bit category set."""
    return [k for k in range(64) if (int(mask) >> k) & 1]


# ----------------------------------------------------------------------------------- datasets

def two_class_gaussian(N: int, F: int, seed: int, frac0: float = 0.37, shift: float = 1.0):
    """Two classes, x|y=0 ~ N(0, I), x|y=1 ~ N(shift * 1, I); n0 = round(frac0 * N), shuffled."""
    rng = np.random.default_rng([seed, 11])
    n0 = int(round(frac0 * N))
    y = np.concatenate([np.zeros(n0, np.int32), np.ones(N - n0, np.int32)])
    rng.shuffle(y)
    X = rng.standard_normal((N, F), dtype=np.float32)
    X += (y[:, None] * np.float32(shift)).astype(np.float32)
    return X, y


def gaussian_mixture(N: int, F: int, K: int, seed: int):
    """K classes with uniform labels, x|y=k ~ N(mu_k, I), mu_k ~ N(0, I)."""
    rng = np.random.default_rng([seed, 12])
    mu = rng.standard_normal((K, F), dtype=np.float32)
    y = rng.integers(0, K, size=N, dtype=np.int32)
    X = rng.standard_normal((N, F), dtype=np.float32)
    X += mu[y]
    return X, y


def categorical_mixture(N: int, F: int, K: int, seed: int, n_cat: int, n_codes: int = 16):
    """The K-class Gaussian mixture with its last ``n_cat`` features categorical: feature j holds
    integer codes 0..n_codes-1 (as float32) drawn per class from a category distribution that
    is itself drawn from a symmetric Dirichlet(1) law, so the codes carry class information."""
    X, y = gaussian_mixture(N, F, K, seed)
    rng = np.random.default_rng([seed, 13])
    probs = rng.dirichlet(np.ones(n_codes), size=(n_cat, K))           # [n_cat, K, n_codes]
    for j in range(n_cat):
        cdf = np.cumsum(probs[j], axis=1)
        u = rng.random(N)
        codes = np.minimum((u[:, None] > cdf[y]).sum(axis=1), n_codes - 1)
        X[:, F - n_cat + j] = codes.astype(np.float32)
    return X, y


def quantile_table(X: np.ndarray, m: int = 65536) -> np.ndarray:
    """Per-feature sorted sample (F x m') used to draw thresholds at empirical quantiles."""
    sub = X[: min(len(X), m)]
    return np.sort(sub, axis=0).T.copy()


# ---------------------------------------------------------------------------------- rule sets

def random_rulesets(qtab: np.ndarray, K: int, P: int, R, C, seed: int, pair_prob: float = 0.2,
                    default=None, cat_from: int | None = None, n_codes: int = 16) -> Batch:
    """Random ordered rule sets.

    R and C are either an int (fixed) or an inclusive (lo, hi) range drawn uniformly per set / rule.
    Conditions: PAIR with probability ``pair_prob``; op uniform over {'>', '<'}; a, b ~ U[-1, 1];
    a threshold t = fl32(a * Q_f(q)) with q ~ U(0.05, 0.95) and Q_f the lower empirical quantile
    of feature f.  Rule class ~ U{0..K-1}.  ``default`` is an int (one class for all sets) or None
    (uniform per set).  With ``cat_from``, features f >= cat_from are categorical (codes
    0..n_codes-1): a condition on such a feature is a membership test of a random non-empty set
    of codes (each code in with probability 1/2), and a pair whose second feature is categorical
    becomes a threshold condition on its first.
    """
    rng = np.random.default_rng([seed, 21])
    F, m = qtab.shape

    def draw(spec, size):
        if isinstance(spec, (int, np.integer)):
            return np.full(size, int(spec), np.int64)
        lo, hi = spec
        return rng.integers(lo, hi + 1, size=size)

    Rp = draw(R, P)
    R_tot = int(Rp.sum())
    Cr = draw(C, R_tot)
    C_tot = int(Cr.sum())
    set_rule_off = np.zeros(P + 1, np.int32)
    set_rule_off[1:] = np.cumsum(Rp)
    rule_cond_off = np.zeros(R_tot + 1, np.int32)
    rule_cond_off[1:] = np.cumsum(Cr)
    rule_class = rng.integers(0, K, size=R_tot, dtype=np.int32)
    if default is None:
        set_default = rng.integers(0, K, size=P, dtype=np.int32)
    else:
        set_default = np.full(P, int(default), np.int32)

    is_pair = rng.random(C_tot) < pair_prob
    cond_f = rng.integers(0, F, size=C_tot, dtype=np.int32)
    g = rng.integers(0, F - 1, size=C_tot, dtype=np.int32) if F > 1 else np.zeros(C_tot, np.int32)
    g = np.where(g >= cond_f, g + 1, g) if F > 1 else g        # g != f
    cond_g = np.where(is_pair, g, -1).astype(np.int32)
    cond_op = rng.integers(0, 2, size=C_tot).astype(np.int8)
    cond_a = rng.uniform(-1.0, 1.0, size=C_tot).astype(np.float32)
    cond_b = np.where(is_pair, rng.uniform(-1.0, 1.0, size=C_tot), 0.0).astype(np.float32)
    q = rng.uniform(0.05, 0.95, size=C_tot)
    qidx = np.floor(q * (m - 1)).astype(np.int64)
    Q = qtab[cond_f, qidx]
    cond_t = np.where(is_pair, np.float32(0), cond_a * Q).astype(np.float32)
    cond_set = None
    if cat_from is not None:
        is_cat = cond_f >= cat_from
        to_thr = ~is_cat & (cond_g >= cat_from)
        cond_g = np.where(is_cat | to_thr, -1, cond_g).astype(np.int32)
        cond_b = np.where(is_cat | to_thr, 0.0, cond_b).astype(np.float32)
        cond_t = np.where(to_thr, cond_a * Q, cond_t).astype(np.float32)
        cond_t = np.where(is_cat, 0.0, cond_t).astype(np.float32)
        cond_a = np.where(is_cat, 0.0, cond_a).astype(np.float32)
        cond_op = np.where(is_cat, IN, cond_op).astype(np.int8)
        bits = rng.random((C_tot, n_codes)) < 0.5
        bits[np.arange(C_tot), rng.integers(0, n_codes, size=C_tot)] = True      # non-empty
        masks = (bits.astype(np.uint64) << np.arange(n_codes, dtype=np.uint64)).sum(axis=1, dtype=np.uint64)
        cond_set = np.where(is_cat, masks, np.uint64(0)).astype(np.uint64)
    return Batch(set_rule_off, rule_cond_off, rule_class, set_default, cond_f, cond_g, cond_op,
                 cond_a, cond_b, cond_t, cond_set)


def majority_class(y: np.ndarray, K: int) -> int:
    return int(np.argmax(np.bincount(y, minlength=K)))   # ties -> lowest id


# ---------------------------------------------------------------------------------- workloads

@dataclasses.dataclass
class Workload:
    name: str
    X: np.ndarray
    y: np.ndarray
    K: int
    batch: Batch
    tau: float = 0.1

    @property
    def N(self):
        return int(self.X.shape[0])

    @property
    def F(self):
        return int(self.X.shape[1])

    def nominal_cond_evals(self) -> int:
        return self.batch.nominal_conditions() * self.N


def plain_hard(seed: int = 0, N: int = 569, F: int = 30, P: int = 64) -> Workload:
    """P=64 sets x R=8 rules x C~U{1..3}; N=569 x F=30, two classes 37/63, mean shift 1.0."""
    X, y = two_class_gaussian(N, F, seed)
    b = random_rulesets(quantile_table(X), 2, P, 8, (1, 3), seed, default=majority_class(y, 2))
    return Workload(f"plain-hard P={P} R=8 C=1..3 N={N} F={F} K=2", X, y, 2, b)


def ragged_hard(seed: int = 0, N: int = 1 << 20, F: int = 128, P: int = 4096, K: int = 10) -> Workload:
    """P=4096 sets, R~U{1..64}, C~U{1..8}; N=2^20 x F=128, 10-class Gaussian mixture."""
    X, y = gaussian_mixture(N, F, K, seed)
    b = random_rulesets(quantile_table(X), K, P, (1, 64), (1, 8), seed, default=None)
    return Workload(f"ragged-hard P={P} R=1..64 C=1..8 N={N} F={F} K={K}", X, y, K, b)


def soft_tune(seed: int = 0, N: int = 262144, F: int = 64, P: int = 1024, R: int = 32, C: int = 4) -> Workload:
    """P=1024 x R=32 x C=4; N=262144 x F=64, two classes; tau = 0.1."""
    X, y = two_class_gaussian(N, F, seed)
    b = random_rulesets(quantile_table(X), 2, P, R, C, seed, default=majority_class(y, 2))
    return Workload(f"soft-tune P={P} R={R} C={C} N={N} F={F} K=2 tau=0.1", X, y, 2, b, tau=0.1)


def evolution_data(seed: int = 0, N: int = 100000, F: int = 32):
    """The binary task of the device-resident evolution loop: N=100000 x F=32, two classes."""
    return two_class_gaussian(N, F, seed)


def serving_runs(seed: int = 0, runs: int = 256):
    """Per-run dataset shapes of the serving workload: N log-uniform [500, 500000],
    F ~ U{8..256}, K ~ U{2..10}."""
    rng = np.random.default_rng([seed, 31])
    N = np.exp(rng.uniform(np.log(500), np.log(500000), size=runs)).astype(np.int64)
    F = rng.integers(8, 257, size=runs)
    K = rng.integers(2, 11, size=runs)
    return N, F, K


def serving_request_sizes(seed: int, count: int):
    """Per-request population sizes: P log-uniform [16, 2048]."""
    rng = np.random.default_rng([seed, 32])
    return np.exp(rng.uniform(np.log(16), np.log(2048), size=count)).astype(np.int64)


def boundary_samples(batch: Batch, F: int, N: int, seed: int, frac: float = 0.7, ulps: int = 2):
    """Samples crowded onto condition boundaries, for exact-compare tests.

    For a random condition, feature f gets a value whose product with ``a`` lands on, or a few
    float32 ulps beside, the right-hand side (t, or the product b*x[g] for a pair condition);
    the remaining features are standard normal. A fraction ``frac`` of samples is built this way.
    """
    rng = np.random.default_rng([seed, 41])
    X = rng.standard_normal((N, F)).astype(np.float32)
    C = batch.C
    if C == 0:
        return X
    for n in range(N):
        if rng.random() >= frac:
            continue
        for _ in range(int(rng.integers(1, 4))):
            c = int(rng.integers(0, C))
            f, g = int(batch.cond_f[c]), int(batch.cond_g[c])
            a = np.float32(batch.cond_a[c])
            if a == 0:
                continue
            if g >= 0 and g != f:
                rhs = np.float32(batch.cond_b[c]) * X[n, g]
            else:
                rhs = np.float32(batch.cond_t[c])
            x = np.float32(np.float64(rhs) / np.float64(a))
            k = int(rng.integers(-ulps, ulps + 1))
            direction = np.float32(np.inf) if k > 0 else np.float32(-np.inf)
            for _ in range(abs(k)):
                x = np.nextafter(x, direction, dtype=np.float32)
            X[n, f] = x
    return X


# ------------------------------------------------------------------------------ populations

POP_FIELDS = ("nrule", "deflt", "rcls", "ncond", "cf", "cg", "cop", "ca", "cb", "ct")


def population_from_batch(batch: Batch, RMAX: int, CMAX: int):
    """Fixed-slot population arrays (rule r of set p at [p, r], condition k at [p, r, k]) from a
    CSR batch whose sets have <= RMAX rules of 1..CMAX conditions. Unused slots are zero."""
    P = batch.P
    pop = {"nrule": np.zeros(P, np.int32), "deflt": batch.set_default.astype(np.int32).copy(),
           "rcls": np.zeros((P, RMAX), np.int32), "ncond": np.zeros((P, RMAX), np.int32),
           "cf": np.zeros((P, RMAX, CMAX), np.int32), "cg": np.full((P, RMAX, CMAX), -1, np.int32),
           "cop": np.zeros((P, RMAX, CMAX), np.int8), "ca": np.zeros((P, RMAX, CMAX), np.float32),
           "cb": np.zeros((P, RMAX, CMAX), np.float32), "ct": np.zeros((P, RMAX, CMAX), np.float32)}
    for p in range(P):
        r0, r1 = batch.set_rule_off[p], batch.set_rule_off[p + 1]
        assert r1 - r0 <= RMAX
        pop["nrule"][p] = r1 - r0
        for j, r in enumerate(range(r0, r1)):
            c0, c1 = batch.rule_cond_off[r], batch.rule_cond_off[r + 1]
            assert 1 <= c1 - c0 <= CMAX
            pop["rcls"][p, j] = batch.rule_class[r]
            pop["ncond"][p, j] = c1 - c0
            sl = slice(c0, c1)
            pop["cf"][p, j, :c1 - c0] = batch.cond_f[sl]
            pop["cg"][p, j, :c1 - c0] = batch.cond_g[sl]
            pop["cop"][p, j, :c1 - c0] = batch.cond_op[sl]
            pop["ca"][p, j, :c1 - c0] = batch.cond_a[sl]
            pop["cb"][p, j, :c1 - c0] = batch.cond_b[sl]
            pop["ct"][p, j, :c1 - c0] = batch.cond_t[sl]
    return pop


def batch_from_population(pop) -> Batch:
    """CSR batch of the live slots of a fixed-slot population."""
    P, RMAX, CMAX = pop["cf"].shape
    nrule = pop["nrule"]
    set_rule_off = np.zeros(P + 1, np.int32)
    set_rule_off[1:] = np.cumsum(nrule)
    live = np.arange(RMAX)[None, :] < nrule[:, None]
    nc = pop["ncond"][live]
    rule_cond_off = np.zeros(len(nc) + 1, np.int32)
    rule_cond_off[1:] = np.cumsum(nc)
    cmask = live[:, :, None] & (np.arange(CMAX)[None, None, :] < pop["ncond"][:, :, None])
    return Batch(set_rule_off, rule_cond_off, pop["rcls"][live].astype(np.int32),
                 pop["deflt"].astype(np.int32), pop["cf"][cmask].astype(np.int32),
                 pop["cg"][cmask].astype(np.int32), pop["cop"][cmask].astype(np.int8),
                 pop["ca"][cmask].astype(np.float32), pop["cb"][cmask].astype(np.float32),
                 pop["ct"][cmask].astype(np.float32))


def initial_population(X, y, K, P, RMAX=32, CMAX=6, seed=0):
    """Random initial population: R ~ U{1..RMAX}, C ~ U{1..CMAX}, default = majority class."""
    b = random_rulesets(quantile_table(X), K, P, (1, RMAX), (1, CMAX), seed,
                        default=majority_class(y, K))
    return population_from_batch(b, RMAX, CMAX)
