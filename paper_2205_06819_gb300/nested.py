"""Nested sampling driver on the batched likelihood (Sec. 2.5; Skilling 2004) with a slice-
sampling proposal (Neal 2003, the proposal the paper selects) and batched replacement of
live points.

What the paper describes: N live points are drawn from the prior; at each iteration the
live point of lowest likelihood L* is discarded, the prior mass enclosed by the likelihood
contour shrinks as X_i = t_i X_{i-1} with t_i the largest of N uniform numbers (so the
expected log shrinkage is 1/N), the evidence grows by L* (X_{i-1} - X_i), and the point is
replaced by a new draw from the prior restricted to L > L*.  Sampling stops once the live
points can no longer change Z by more than a chosen fraction.

Batching, so that one likelihood call evaluates many models: the K worst live points are
discarded together.  Discarding them one after another from N, N-1, ..., N-K+1 live points
shrinks ln X by 1/N, 1/(N-1), ..., 1/(N-K+1) in turn; the K replacements are then drawn at
once, each from an independent constrained slice-sampling chain started at a randomly
chosen surviving live point, so the likelihood sees batches of K (fewer as chains finish).
The contour for the whole batch is the largest discarded likelihood.

Each chain step is a hit-and-run slice step in the unit cube: a direction from the live
points' covariance (scaled to about the radius of the live set), an interval one such
step long placed at random around the current point, stepped out while its ends stay inside the contour, then shrunk towards the
current point until a uniform draw from it lies inside (Neal 2003, Sec. 4).  Points outside
the cube are outside the prior support and count as outside the contour.

The sampler runs on the host in float64 with a seeded PCG64 generator; its state can be
saved and resumed bit for bit.  ``loglike`` maps theta [B, P] float64 (numpy) to logL [B];
``gpu_loglike`` adapts a ``model.Model`` to that form.
"""
from __future__ import annotations

import math
import pickle
from dataclasses import dataclass

import numpy as np


@dataclass
class NestedResult:
    logz: float                  # ln Z
    logz_err: float              # sqrt(H / N)
    information: float           # H [nats]
    n_iter: int                  # batch iterations
    n_dead: int                  # discarded points (excluding the final live set)
    n_like: int                  # likelihood evaluations
    samples: np.ndarray          # [n, P] theta of the dead points, then the final live points
    log_weights: np.ndarray      # [n] ln(posterior weight), normalised to sum 1
    log_l: np.ndarray            # [n]

    def equal_weight_samples(self, seed: int = 0) -> np.ndarray:
        """Rows resampled with probability equal to their posterior weight (systematic
        resampling, so the count of each row differs from n w_i by less than one)."""
        w = np.exp(self.log_weights - self.log_weights.max())
        w /= w.sum()
        n = len(w)
        rng = np.random.Generator(np.random.PCG64(seed))
        pos = (rng.random() + np.arange(n)) / n
        idx = np.minimum(np.searchsorted(np.cumsum(w), pos), n - 1)
        return self.samples[idx]

    def quantiles(self, q) -> np.ndarray:
        """Weighted posterior quantiles [len(q), P] (the paper quotes the median and the
        16th / 84th percentiles)."""
        w = np.exp(self.log_weights - self.log_weights.max())
        q = np.atleast_1d(np.asarray(q, dtype=np.float64))
        out = np.empty((len(q), self.samples.shape[1]))
        for j in range(self.samples.shape[1]):
            o = np.argsort(self.samples[:, j], kind="stable")
            c = np.cumsum(w[o])
            c = (c - 0.5 * w[o]) / c[-1]
            out[:, j] = np.interp(q, c, self.samples[o, j])
        return out

    def mean_cov(self):
        w = np.exp(self.log_weights - self.log_weights.max())
        w /= w.sum()
        m = w @ self.samples
        d = self.samples - m
        return m, (d * w[:, None]).T @ d


class BoxPrior:
    """Uniform prior on a box [P, 2] (lo == hi fixes a slot), with optional slots uniform in
    log10 and an inclination slot uniform in sin i (the solid-angle prior of Sec. 3.1).
    The sampler moves in the unit cube of the free slots only."""

    def __init__(self, box, sin_slot: int | None = None, log_slots=()):
        self.box = np.asarray(box, dtype=np.float64)
        self.free = np.flatnonzero(self.box[:, 1] > self.box[:, 0])
        self.ndim = len(self.free)
        self.sin_slot, self.log_slots = sin_slot, tuple(log_slots)

    def __call__(self, u: np.ndarray) -> np.ndarray:
        u = np.atleast_2d(u)
        th = np.repeat(self.box[None, :, 0], u.shape[0], axis=0)
        lo, hi = self.box[self.free, 0], self.box[self.free, 1]
        th[:, self.free] = lo + u * (hi - lo)
        for s in self.log_slots:
            if s in self.free:
                k = int(np.flatnonzero(self.free == s)[0])
                a, b = math.log10(self.box[s, 0]), math.log10(self.box[s, 1])
                th[:, s] = 10.0 ** (a + u[:, k] * (b - a))
        if self.sin_slot is not None and self.sin_slot in self.free:
            k = int(np.flatnonzero(self.free == self.sin_slot)[0])
            s0, s1 = math.sin(self.box[self.sin_slot, 0]), math.sin(self.box[self.sin_slot, 1])
            th[:, self.sin_slot] = np.arcsin(s0 + u[:, k] * (s1 - s0))
        return th


def gpu_loglike(model, gal_idx: int | None = None):
    """theta [B, P] float64 (host) -> logL [B] float64 through bang_loglike_batch (see
    _GpuLogLike)."""
    return _GpuLogLike(model, gal_idx)


def _bucket(n: int) -> int:
    """Call size for n rows: the next of 16, 20, 28, 36, 48, 60, 76, 96, ... (each 5/4 of
    the one before, rounded up to a multiple of 4), so that a sampler's calls come in a few
    dozen sizes whose plans and captured graphs the library keeps."""
    b = 16
    while b < n:
        b = (b * 5 // 4 + 3) // 4 * 4
    return b


class _GpuLogLike:
    """theta [B, P] float64 (host) -> logL [B] float64 through bang_loglike_batch (host
    buffers: the library stages them).  Every call is padded to a bucket size (_bucket) with
    copies of its first row, whose values are dropped: the sampler's calls vary in size from
    one step to the next, and the library keeps a plan and a captured graph per size."""

    def __init__(self, model, gal_idx: int | None = None):
        import torch
        self._torch, self.model, self.gal_idx = torch, model, gal_idx

    def __call__(self, theta: np.ndarray) -> np.ndarray:
        n = len(theta)
        if n == 0:
            return np.empty(0)
        th = np.ascontiguousarray(theta, dtype=np.float32)
        nb = _bucket(n)
        if nb > n:
            th = np.concatenate([th, np.repeat(th[:1], nb - n, axis=0)])
        gi = None if self.gal_idx is None else np.full(nb, self.gal_idx, dtype=np.int32)
        return self.model.loglike(self._torch.from_numpy(th), gal_idx=gi).numpy()[:n]


def _logaddexp(a: float, b: float) -> float:
    if a == -math.inf:
        return b
    if b == -math.inf:
        return a
    m = max(a, b)
    return m + math.log(math.exp(a - m) + math.exp(b - m))


class NestedSampler:
    """Batched nested sampling over the unit cube of ``prior.ndim`` free parameters.

    n_live       live points N
    batch        points K discarded and replaced per iteration (1 <= K < N)
    slice_steps  hit-and-run slice steps per replacement chain (default max(10, 3 P)): too
                 few leave the new points correlated with their starting points, which biases
                 ln Z high when K is a large share of N
    frac         stop once L_max X < frac Z (the remaining live points can change Z by less
                 than this fraction)
    speculate    positions per chain evaluated in one likelihood call during step-out and
                 shrinking (1: one at a time).  With m > 1 each chain's next m step-out
                 positions, and its next m shrink candidates drawn as if each earlier one
                 were rejected, go into one call and the first outcome that ends the search
                 is taken: the same sequence the one-at-a-time procedure draws, so the
                 chain's distribution is unchanged; the candidates after it are evaluated
                 and discarded.  Fewer, larger calls: worth it when a call's latency, not
                 its rows, sets its cost.
    """

    def __init__(self, loglike, prior, n_live: int = 400, batch: int = 40, slice_steps: int | None = None,
                 frac: float = 0.01, seed: int = 0, max_iter: int = 1_000_000,
                 max_steps_out: int = 16, max_shrink: int = 64, speculate: int = 1):
        if not 1 <= batch < n_live:
            raise ValueError("need 1 <= batch < n_live")
        if prior.ndim < 1:
            raise ValueError("the prior has no free parameter")
        self.loglike, self.prior = loglike, prior
        self.ndim, self.n_live, self.batch = prior.ndim, n_live, batch
        self.slice_steps = slice_steps if slice_steps is not None else max(10, 3 * prior.ndim)
        self.frac, self.max_iter = frac, max_iter
        self.max_steps_out, self.max_shrink = max_steps_out, max_shrink
        if speculate < 1:
            raise ValueError("need speculate >= 1")
        self.speculate = int(speculate)
        self.rng = np.random.Generator(np.random.PCG64(seed))
        self.n_like = 0
        self.it = 0
        self.plateau = False
        self.logz, self.h, self.logx = -math.inf, 0.0, 0.0
        self.dead_u, self.dead_l, self.dead_lw = [], [], []
        self.u = self.rng.random((n_live, self.ndim))
        self.lv = self._logl(self.u)

    # -- likelihood --------------------------------------------------------------------
    def _logl(self, u: np.ndarray) -> np.ndarray:
        if len(u) == 0:
            return np.empty(0)
        self.n_like += len(u)
        out = np.asarray(self.loglike(self.prior(u)), dtype=np.float64).reshape(len(u))
        return np.where(np.isnan(out), -np.inf, out)

    def _above(self, pts: np.ndarray, lstar: float):
        """(inside, logL): points outside the cube are outside the prior support and are not
        evaluated."""
        lp = self._eval(pts)
        return lp > lstar, lp

    # -- evidence bookkeeping ----------------------------------------------------------
    def _add(self, logl: float, log_width: float):
        lwt = logl + log_width
        self.dead_lw.append(lwt)
        if lwt == -math.inf:
            return
        logz_new = _logaddexp(self.logz, lwt)
        carried = math.exp(self.logz - logz_new) * (self.h + self.logz) if self.logz > -math.inf else 0.0
        self.h = math.exp(lwt - logz_new) * logl + carried - logz_new
        self.logz = logz_new

    # -- replacement chains ------------------------------------------------------------
    def _chains(self, u: np.ndarray, lu: np.ndarray, lstar: float, chol: np.ndarray):
        if self.speculate > 1:
            return self._chains_speculative(u, lu, lstar, chol)
        K, D = u.shape
        width = 0.5 * math.sqrt(D + 2.0)
        for _ in range(self.slice_steps):
            z = self.rng.standard_normal((K, D))
            z /= np.linalg.norm(z, axis=1, keepdims=True)
            d = (z @ chol.T) * width
            r = self.rng.random(K)
            lo, hi = -r, 1.0 - r
            act_lo, act_hi = np.ones(K, bool), np.ones(K, bool)
            for _ in range(self.max_steps_out):
                if not (act_lo.any() or act_hi.any()):
                    break
                pts = np.concatenate([u[act_lo] + lo[act_lo, None] * d[act_lo],
                                      u[act_hi] + hi[act_hi, None] * d[act_hi]])
                ok, _ = self._above(pts, lstar)
                n_lo = int(act_lo.sum())
                g_lo, g_hi = np.zeros(K, bool), np.zeros(K, bool)
                g_lo[act_lo], g_hi[act_hi] = ok[:n_lo], ok[n_lo:]
                lo[g_lo] -= 1.0
                hi[g_hi] += 1.0
                act_lo, act_hi = g_lo, g_hi
            done = np.zeros(K, bool)
            for _ in range(self.max_shrink):
                t = lo + self.rng.random(K) * (hi - lo)
                todo = ~done
                cand = u[todo] + t[todo, None] * d[todo]
                ok, lp = self._above(cand, lstar)
                idx = np.flatnonzero(todo)
                acc = idx[ok]
                u[acc], lu[acc] = cand[ok], lp[ok]
                done[acc] = True
                rej = idx[~ok]
                neg = rej[t[rej] < 0.0]
                pos = rej[t[rej] >= 0.0]
                lo[neg], hi[pos] = t[neg], t[pos]
                if done.all():
                    break
        return u, lu

    def _chains_speculative(self, u: np.ndarray, lu: np.ndarray, lstar: float, chol: np.ndarray):
        """_chains with ``speculate`` positions per chain and call (see the class notes)."""
        gen = self._chain_gen(u, lu, lstar, chol)
        try:
            pts = next(gen)
            while True:
                pts = gen.send(self._eval(pts))
        except StopIteration as stop:
            return stop.value

    def _eval(self, pts: np.ndarray) -> np.ndarray:
        """logL of pts, -inf outside the unit cube (the prior's support; not evaluated)."""
        inc = np.all((pts >= 0.0) & (pts <= 1.0), axis=1)
        lp = np.full(len(pts), -np.inf)
        lp[inc] = self._logl(pts[inc])
        return lp

    def _chain_gen(self, u: np.ndarray, lu: np.ndarray, lstar: float, chol: np.ndarray):
        """The speculative chains as a generator: yields the points of each likelihood call,
        receives their logL (-inf outside the cube) and returns (u, lu) at the end."""
        K, D = u.shape
        m = self.speculate
        width = 0.5 * math.sqrt(D + 2.0)
        for _ in range(self.slice_steps):
            z = self.rng.standard_normal((K, D))
            z /= np.linalg.norm(z, axis=1, keepdims=True)
            d = (z @ chol.T) * width
            r = self.rng.random(K)
            lo, hi = -r, 1.0 - r
            # step out: positions lo, lo - 1, ..., lo - (m - 1) (and hi upwards) at once; an
            # end stops at its first position outside the contour
            act_lo, act_hi = np.ones(K, bool), np.ones(K, bool)
            used = 0
            while used < self.max_steps_out and (act_lo.any() or act_hi.any()):
                mm = min(m, self.max_steps_out - used)
                il, ih = np.flatnonzero(act_lo), np.flatnonzero(act_hi)
                offs = np.arange(mm, dtype=np.float64)
                pl = lo[il, None] - offs[None, :]
                ph = hi[ih, None] + offs[None, :]
                pts = np.concatenate([(u[il, None, :] + pl[..., None] * d[il, None, :]).reshape(-1, D),
                                      (u[ih, None, :] + ph[..., None] * d[ih, None, :]).reshape(-1, D)])
                ok = (yield pts) > lstar
                okl = ok[:len(il) * mm].reshape(len(il), mm)
                okh = ok[len(il) * mm:].reshape(len(ih), mm)
                fl = np.where(okl.all(axis=1), mm, np.argmin(okl, axis=1))
                fh = np.where(okh.all(axis=1), mm, np.argmin(okh, axis=1))
                lo[il] -= fl
                hi[ih] += fh
                act_lo = np.zeros(K, bool)
                act_hi = np.zeros(K, bool)
                act_lo[il[fl == mm]] = True
                act_hi[ih[fh == mm]] = True
                used += mm
            # shrink: the next m candidates of each open chain, each drawn from the interval
            # the earlier ones would leave if rejected; the first inside the contour is taken
            done = np.zeros(K, bool)
            used = 0
            while used < self.max_shrink and not done.all():
                mm = min(m, self.max_shrink - used)
                idx = np.flatnonzero(~done)
                n = len(idx)
                lo_c, hi_c = lo[idx].copy(), hi[idx].copy()
                draws = self.rng.random((n, mm))
                ts = np.empty((n, mm))
                for j in range(mm):
                    t = lo_c + draws[:, j] * (hi_c - lo_c)
                    ts[:, j] = t
                    neg = t < 0.0
                    lo_c = np.where(neg, t, lo_c)
                    hi_c = np.where(neg, hi_c, t)
                cand = u[idx, None, :] + ts[..., None] * d[idx, None, :]
                lp = (yield cand.reshape(-1, D)).reshape(n, mm)
                ok = lp > lstar
                hit = ok.any(axis=1)
                first = np.argmax(ok, axis=1)
                acc = idx[hit]
                u[acc] = cand[hit, first[hit]]
                lu[acc] = lp[hit, first[hit]]
                done[acc] = True
                miss = idx[~hit]
                lo[miss], hi[miss] = lo_c[~hit], hi_c[~hit]
                used += mm
        return u, lu

    # -- iteration ---------------------------------------------------------------------
    def converged(self) -> bool:
        if self.plateau:
            return True
        if self.logz == -math.inf:
            return False
        return float(self.lv.max()) + self.logx < self.logz + math.log(self.frac)

    def step(self):
        N, K = self.n_live, self.batch
        order = np.argsort(self.lv, kind="stable")
        worst, keep = order[:K], order[K:]
        lstar = float(self.lv[worst[-1]])
        alive = keep[self.lv[keep] > lstar]
        if len(alive) == 0:
            # a likelihood plateau holds every live point: the rest of the prior mass has
            # the same L, which the final live share already counts
            self.plateau = True
            return
        for k in range(K):
            shrink = 1.0 / (N - k)
            self._add(float(self.lv[worst[k]]), self.logx + math.log(-math.expm1(-shrink)))
            self.logx -= shrink
        self.dead_u.append(self.u[worst].copy())
        self.dead_l.append(self.lv[worst].copy())
        start = alive[self.rng.integers(0, len(alive), K)]
        cov = np.atleast_2d(np.cov(self.u[keep].T))
        cov += np.eye(self.ndim) * (1e-12 + 1e-9 * np.trace(cov) / self.ndim)
        chol = np.linalg.cholesky(cov)
        nu, nl = self._chains(self.u[start].copy(), self.lv[start].copy(), lstar, chol)
        self.u[worst], self.lv[worst] = nu, nl
        self.it += 1

    def run(self, checkpoint: str | None = None, every: int = 50, max_iter: int | None = None) -> NestedResult:
        """Iterate until converged (or ``max_iter`` more iterations); with ``checkpoint``,
        save the state there every ``every`` iterations and at the end."""
        stop = self.it + (max_iter if max_iter is not None else self.max_iter)
        while not self.converged() and self.it < stop:
            self.step()
            if checkpoint and self.it % every == 0:
                self.save(checkpoint)
        if checkpoint:
            self.save(checkpoint)
        return self.result()

    def result(self) -> NestedResult:
        """Dead points plus the final live points, each live point given X / N."""
        N = self.n_live
        saved = (self.logz, self.h, list(self.dead_lw))
        for k in np.argsort(self.lv, kind="stable"):
            self._add(float(self.lv[k]), self.logx - math.log(N))
        lw = np.array(self.dead_lw)
        logz_f, h_f = self.logz, self.h
        self.logz, self.h, self.dead_lw = saved
        u = np.concatenate(self.dead_u + [self.u[np.argsort(self.lv, kind="stable")]])
        ll = np.concatenate(self.dead_l + [np.sort(self.lv, kind="stable")])
        return NestedResult(logz=logz_f, logz_err=math.sqrt(max(h_f, 0.0) / N), information=h_f,
                            n_iter=self.it, n_dead=len(lw) - N, n_like=self.n_like,
                            samples=self.prior(u), log_weights=lw - logz_f, log_l=ll)

    # -- checkpoint / resume -----------------------------------------------------------
    _STATE = ("n_live", "batch", "slice_steps", "frac", "max_steps_out", "max_shrink", "speculate", "n_like",
              "it", "plateau", "logz", "h", "logx", "dead_u", "dead_l", "dead_lw", "u", "lv")
    _DEFAULTS = {"speculate": 1}   # states saved before this option: one position at a time

    def state_dict(self) -> dict:
        s = {k: getattr(self, k) for k in self._STATE}
        s["rng"] = self.rng.bit_generator.state
        return pickle.loads(pickle.dumps(s))

    def load_state_dict(self, s: dict):
        for k in self._STATE:
            setattr(self, k, s.get(k, self._DEFAULTS[k]) if k in self._DEFAULTS else s[k])
        self.ndim = self.u.shape[1]
        self.rng.bit_generator.state = s["rng"]

    def save(self, path: str):
        import os
        tmp = path + ".tmp"
        with open(tmp, "wb") as f:
            pickle.dump(self.state_dict(), f)
        os.replace(tmp, path)

    @classmethod
    def resume(cls, path: str, loglike, prior, max_iter: int = 1_000_000) -> "NestedSampler":
        with open(path, "rb") as f:
            s = pickle.load(f)
        self = cls.__new__(cls)
        self.loglike, self.prior, self.max_iter = loglike, prior, max_iter
        self.rng = np.random.Generator(np.random.PCG64(0))
        self.load_state_dict(s)
        return self
