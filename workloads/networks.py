"""Reaction networks of the paper's models and a synthetic large network shaped like FceRI.

Each network is a plain list of reactions: reactants and products as (species, multiplicity)
pairs, a rate constant per reaction (one row per parameter set for batched sweeps), an optional
Hill-repression law, and the species held at a constant count.  How propensities follow from
these is the business of the code that consumes them, not of this module.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

MASS_ACTION = 0
HILL_REPRESSION = 1


@dataclass
class NetworkSpec:
    """A reaction network.  ``rate`` has shape (n_param_sets, n_reactions)."""

    species: list[str]
    reactants: list[list[tuple[int, int]]]
    products: list[list[tuple[int, int]]]
    rate: np.ndarray
    rate_law: np.ndarray = None
    hill_species: np.ndarray = None
    hill_K: np.ndarray = None
    hill_n: np.ndarray = None
    fixed_count: np.ndarray = None
    name: str = ""
    notes: dict = field(default_factory=dict)

    def __post_init__(self):
        M = len(self.reactants)
        assert len(self.products) == M
        self.rate = np.atleast_2d(np.asarray(self.rate, dtype=np.float64))
        assert self.rate.shape[1] == M
        if self.rate_law is None:
            self.rate_law = np.zeros(M, dtype=np.int32)
        self.rate_law = np.asarray(self.rate_law, dtype=np.int32)
        if self.hill_species is None:
            self.hill_species = np.zeros(M, dtype=np.int32)
        self.hill_species = np.asarray(self.hill_species, dtype=np.int32)
        if self.hill_K is None:
            self.hill_K = np.ones((1, M), dtype=np.float64)
        self.hill_K = np.atleast_2d(np.asarray(self.hill_K, dtype=np.float64))
        if self.hill_n is None:
            self.hill_n = np.ones(M, dtype=np.int32)
        self.hill_n = np.asarray(self.hill_n, dtype=np.int32)
        if self.fixed_count is None:
            self.fixed_count = np.full(self.n_species, -1, dtype=np.int32)
        self.fixed_count = np.asarray(self.fixed_count, dtype=np.int32)

    @property
    def n_species(self) -> int:
        return len(self.species)

    @property
    def n_reactions(self) -> int:
        return len(self.reactants)

    @property
    def n_param_sets(self) -> int:
        return self.rate.shape[0]

    def csr(self) -> dict:
        """Reactant/product lists as CSR int32 arrays."""
        def pack(lists):
            ptr = np.zeros(len(lists) + 1, dtype=np.int32)
            sp, mu = [], []
            for j, lst in enumerate(lists):
                for s, m in lst:
                    sp.append(s)
                    mu.append(m)
                ptr[j + 1] = len(sp)
            return ptr, np.asarray(sp, dtype=np.int32), np.asarray(mu, dtype=np.int32)

        rp, rs, rm = pack(self.reactants)
        pp, ps, pm = pack(self.products)
        return dict(reac_ptr=rp, reac_species=rs, reac_mult=rm,
                    prod_ptr=pp, prod_species=ps, prod_mult=pm)

    def hill_K_row(self, p: int) -> np.ndarray:
        return self.hill_K[p % self.hill_K.shape[0]]


def birth_death(kb: float = 10.0, kd: float = 0.1) -> NetworkSpec:
    """0 -> X at rate kb, X -> 0 at kd per molecule (stationary law Poisson(kb/kd))."""
    return NetworkSpec(species=["X"], reactants=[[], [(0, 1)]], products=[[(0, 1)], []],
                       rate=[[kb, kd]], name="birth_death")


def schlogl(c1=3e-7, c2=1e-4, c3=1e-3, c4=3.5, A=100000, B=200000) -> NetworkSpec:
    """Schloegl model, Sec. III.B.1 (Eq. "schlogl"): A+2X <-> 3X, B <-> X, A and B constant."""
    X, Ai, Bi = 0, 1, 2
    return NetworkSpec(
        species=["X", "A", "B"],
        reactants=[[(Ai, 1), (X, 2)], [(X, 3)], [(Bi, 1)], [(X, 1)]],
        products=[[(X, 3)], [(Ai, 1), (X, 2)], [(X, 1)], [(Bi, 1)]],
        rate=[[c1, c2, c3, c4]],
        fixed_count=np.array([-1, A, B], dtype=np.int32),
        name="schlogl",
    )


def toggle_switch(a_u, a_v, d: float = 1.0, K: float = 1.0, n: int = 2, b0: float = 0.0) -> NetworkSpec:
    """Two mutually repressing genes U, V (shaped like the epigenetic switch of Sec. III.C).

    Reactions: 0->U at a_u/(1+(V/K)^n); 0->V at a_v/(1+(U/K)^n); U->0, V->0 at d per molecule;
    basal 0->U, 0->V at b0.  ``a_u``/``a_v`` may be arrays (one parameter set per entry).
    """
    a_u = np.atleast_1d(np.asarray(a_u, dtype=np.float64))
    a_v = np.atleast_1d(np.asarray(a_v, dtype=np.float64))
    P = len(a_u)
    rate = np.stack([a_u, a_v, np.full(P, d), np.full(P, d), np.full(P, b0), np.full(P, b0)], axis=1)
    return NetworkSpec(
        species=["U", "V"],
        reactants=[[], [], [(0, 1)], [(1, 1)], [], []],
        products=[[(0, 1)], [(1, 1)], [], [], [(0, 1)], [(1, 1)]],
        rate=rate,
        rate_law=np.array([HILL_REPRESSION, HILL_REPRESSION, 0, 0, 0, 0], dtype=np.int32),
        hill_species=np.array([1, 0, 0, 0, 0, 0], dtype=np.int32),
        hill_K=np.full((1, 6), K),
        hill_n=np.array([n, n, 1, 1, 1, 1], dtype=np.int32),
        name="toggle_switch",
    )


def epigenetic_switch(a1=156.0, a2=30.0, n=3, m=1, K1=1.0, K2=1.0, k0=1.0) -> NetworkSpec:
    """The paper's epigenetic switch, Sec. III.C.1: g1 repressed by g2 (Hill n), g2 by g1 (Hill m)."""
    return NetworkSpec(
        species=["g1", "g2"],
        reactants=[[], [(0, 1)], [], [(1, 1)]],
        products=[[(0, 1)], [], [(1, 1)], []],
        rate=[[a1, k0, a2, k0]],
        rate_law=np.array([HILL_REPRESSION, 0, HILL_REPRESSION, 0], dtype=np.int32),
        hill_species=np.array([1, 0, 0, 0], dtype=np.int32),
        hill_K=np.array([[K2, 1.0, K1, 1.0]]),
        hill_n=np.array([n, 1, m, 1], dtype=np.int32),
        name="epigenetic_switch",
    )


def futile_cycle(kf=1.0, ks=0.1) -> NetworkSpec:
    """Enzymatic futile cycle, Sec. III.A.1 (Eq. "futile").  Species order: S1,S2,E1,E2,B1,B2."""
    S1, S2, E1, E2, B1, B2 = range(6)
    return NetworkSpec(
        species=["S1", "S2", "E1", "E2", "B1", "B2"],
        reactants=[[(E1, 1), (S1, 1)], [(B1, 1)], [(B1, 1)], [(E2, 1), (S2, 1)], [(B2, 1)], [(B2, 1)]],
        products=[[(B1, 1)], [(E1, 1), (S1, 1)], [(E1, 1), (S2, 1)], [(B2, 1)], [(E2, 1), (S2, 1)],
                  [(E2, 1), (S1, 1)]],
        rate=[[kf, kf, ks, kf, kf, ks]],
        name="futile_cycle",
    )


def synthetic_large(n_species: int = 354, n_reactions: int = 3680, frac_uni: float = 0.6,
                    seed: int = 7, k_lo: float = 1e-4, k_hi: float = 1e1) -> NetworkSpec:
    """Random mass-action network with the FceRI model's size (354 species, 3680 reactions).

    Only the shape stands in for FceRI (Sec. III.D): 60 % unimolecular and 40 % bimolecular
    reactions, reactants drawn uniformly with replacement (a repeated species is a homodimer),
    as many products as reactants drawn uniformly, rate constants log-uniform in [k_lo, k_hi].
    Every reaction conserves the total molecule count, so counts stay bounded.
    """
    rng = np.random.default_rng(seed)
    n_uni = int(round(frac_uni * n_reactions))
    reactants, products = [], []
    for j in range(n_reactions):
        order = 1 if j < n_uni else 2
        rs = rng.integers(0, n_species, size=order)
        ps = rng.integers(0, n_species, size=order)

        def merge(v):
            d = {}
            for s in v:
                d[int(s)] = d.get(int(s), 0) + 1
            return sorted(d.items())

        reactants.append(merge(rs))
        products.append(merge(ps))
    perm = rng.permutation(n_reactions)
    reactants = [reactants[i] for i in perm]
    products = [products[i] for i in perm]
    rate = np.exp(rng.uniform(np.log(k_lo), np.log(k_hi), size=n_reactions))
    return NetworkSpec(species=[f"s{i}" for i in range(n_species)], reactants=reactants,
                       products=products, rate=rate[None, :], name="synthetic_large",
                       notes=dict(seed=seed))
