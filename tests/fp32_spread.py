"""How far FP32-sized rounding alone moves the oracle's APPGA trajectory.

Used where the FP64 oracle itself does not fix the image to the FP32 parity
tolerance: the GPU's distance from the oracle is then bounded by a stated
multiple of this spread."""
import numpy as np

from oracle import appga_oracle as O


def oracle_fp32_noisy(prob, par, f0, seed, keep=()):
    """The oracle's APPGA run of par.max_iters maps (Eq. 23 with the momentum
    of Eq. 24) from f^0 = f^1 = f0, with a relative perturbation of FP32 size
    (2^-24 N(0,1)) applied to every new iterate.  Returns the final iterate,
    and also a dict map -> iterate for the maps listed in `keep`."""
    lam = prob.em_lambda()
    th = O.thetas_for(par, par.max_iters)
    rng = np.random.default_rng(seed)
    fk, fkm = f0.copy(), f0.copy()
    kept = {}
    for it in range(par.max_iters):
        fn, _ = O.appga_step(prob, fk, fkm, th[it], par, lam)
        fn = fn * (1.0 + 2.0 ** -24 * rng.standard_normal(fn.shape[0]))
        fkm, fk = fk, fn
        if it + 1 in keep:
            kept[it + 1] = fk.copy()
    return (fk, kept) if keep else fk
