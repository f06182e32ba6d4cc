"""Event builders for tests: seeded inputs from ``synth`` plus a signal injected
with the oracle's waveform (the oracle is test infrastructure; the library never
sees it)."""
import numpy as np

import oracle
import synth


def inject(ev: dict, theta=None, scale: float = 1.0) -> dict:
    th = ev["theta_inj"] if theta is None else np.asarray(theta, dtype=np.float64)
    h = np.stack([oracle.strain(th, ev["geom"][d], ev["gmst"], ev["f"]) for d in range(ev["geom"].shape[0])])
    ev["data"] = ev["noise"] + scale * h
    ev["signal"] = h
    return ev


def event(cfg="C1", **kw) -> dict:
    return inject(synth.make_event(cfg, **kw))


def small_event(sites=("H1", "L1", "V1"), T=8.0, f_low=20.0, f_high=512.0) -> dict:
    """A short multi-detector event (a few thousand grid points) for fast checks."""
    return inject(synth.make_event("C2", T=T, f_low=f_low, f_high=f_high, sites=sites))
