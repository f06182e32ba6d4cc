"""The GPU paths the bounds-check test runs, shared by the normal and the
debug-library runs so that their outputs can be compared."""
import numpy as np
import torch

import synth
from tests._events import inject


def run_paths(rb) -> dict:
    out = {}
    for name, kw, B in (("three", dict(T=64.0, f_high=1024.0), 97), ("two", dict(T=64.0, sites=("H1", "L1")), 150),
                        ("one", dict(T=8.0, sites=("V1",), f_high=512.0), 45)):
        ev = inject(synth.make_event("C2", **kw))
        event = rb.Event.from_synth(ev, n_bins=B)
        th = torch.tensor(synth.posterior_box(ev["theta_inj"], 301, seed=5), device="cuda")
        for mode in ("mixed", "mixed_f64phase", "fp64"):
            L, G = rb.loglike_grad(event, th, mode=mode)
            out[f"{name}_{mode}_L"], out[f"{name}_{mode}_G"] = L.cpu().numpy(), G.cpu().numpy()
        event.rebuild(mode="mixed")  # chunk-expanded summary (or the FP64 one for short grids)
        event.rebuild(mode="fp64")   # FP64 from the stored waveform
        L, G = rb.rebuild_loglike_grad(event, th)
        out[f"{name}_rebuild_L"], out[f"{name}_rebuild_G"] = L.cpu().numpy(), G.cpu().numpy()
        D = ev["geom"].shape[0]
        data = [torch.tensor(np.stack([ev["data"][d].real, ev["data"][d].imag], -1)).pin_memory() for d in range(D)]
        psd = [torch.tensor(ev["psd"][d]).pin_memory() for d in range(D)]
        Lh, Gh = np.zeros(301), np.zeros((301, 13))
        rb.rebuild_loglike_grad_host(event, data, psd, th.cpu().numpy(), Lh, Gh)  # host-link read
        out[f"{name}_host_L"], out[f"{name}_host_G"] = Lh, Gh
        z = th.clone()
        z[:, 9], z[:, 12] = torch.cos(th[:, 9]), torch.sin(th[:, 12])
        lo = np.array([0.5, 0.05, -0.5, -0.5, 0.0, 0.0, 1.0, -1.0, 0.0, -1.0, 0.0, 0.0, -1.0])
        hi = np.array([3.0, 1.0, 0.5, 0.5, 5000.0, 5000.0, 100.0, 1.0, 2 * np.pi, 1.0, np.pi, 2 * np.pi, 1.0])
        logp, gz = rb.mala_init(event, z, lo, hi)
        gen = torch.Generator(device="cuda").manual_seed(3)
        xi = torch.randn(301, 13, dtype=torch.float64, device="cuda", generator=gen)
        u = torch.rand(301, dtype=torch.float64, device="cuda", generator=gen)
        rb.mala_step(event, z, logp, gz, np.full(13, 1e-4), lo, hi, xi, u)
        out[f"{name}_mala_z"] = z.cpu().numpy()
        event.free()
    return out
