"""Oracle solves for the GPU parity tests, run side by side in worker
processes.

The full-size references (2048 x 2048, 50 iterations) take the FP64 oracle
about a minute and a half each on one core, so the tests start them in a
pool of 'spawn' processes (a fork after the CUDA context exists can hang)
and collect them when they are needed.  Every job loads the oracle in its own
process and returns plain numpy arrays.  Test infrastructure only."""
from __future__ import annotations

import multiprocessing as mp

import numpy as np


def _lines(O, spec):
    E, d, b, w, L, p = spec
    return O.Lines(E, d, b, w, L=L, pixel=p)


def solve_job(spec, D, n_iter, omega, tol=0.0, T0=None):
    """(T, rho history, kappa history, iterations) of oracle.solve."""
    from oracle import oracle as O
    T, info = O.solve(_lines(O, spec), np.asarray(D, np.float64), T0=T0, n_iter=n_iter,
                      omega=omega, tol=tol)
    return T, info["rho"], info["kappa"], info["iters"]


def forward_job(spec, tau):
    from oracle import oracle as O
    return O.forward(_lines(O, spec), np.asarray(tau, np.float64))


class Pool:
    """A spawn-context process pool; submit() returns an AsyncResult."""

    def __init__(self, workers: int):
        self._pool = mp.get_context("spawn").Pool(workers)

    def submit(self, fn, *args, **kw):
        return self._pool.apply_async(fn, args, kw)

    def close(self):
        self._pool.close()
        self._pool.join()


def solve_window_job(spec, D, n_iter, omega, tol):
    """The oracle solve with its stopping rule, one iteration at a time:
    returns (iterations run k, {k - 1: T, k: T, k + 1: T}, kappa history).
    The iterate after k + 1 iterations is one more iteration from the result
    (for a comparison with a float32 solve that stopped one iteration
    later); every iteration is the same arithmetic as a multi-iteration
    solve's."""
    from oracle import oracle as O
    ln = _lines(O, spec)
    D = np.asarray(D, np.float64)
    T = np.zeros_like(D)
    prev = T.copy()
    kap = []
    k = 0
    while k < n_iter:
        prev = T
        T, info = O.solve(ln, D, T0=T, n_iter=1, omega=omega, tol=0.0)
        kap.append(float(info["kappa"][0]))
        k += 1
        if kap[-1] <= tol:
            break
    nxt, _ = O.solve(ln, D, T0=T, n_iter=1, omega=omega, tol=0.0)
    return k, {k - 1: prev, k: T, k + 1: nxt}, kap
