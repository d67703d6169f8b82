"""algdock_cycle, one iteration of the paper's loop over a whole run ("Equilibration and
production": an HMC move of every replica, then the exchange sweeps of every ladder, then the
snapshot's reduced energies from the components the trial left), with the run's arrays in host
memory or on the device.  Both must repeat, bit for bit, the same cycles made of the separate
calls (algdock_hmc_cycle, algdock_exchange, algdock_reduced_energies) on device buffers."""
import numpy as np
import pytest

from paper_1507_03703_gb300 import synthetic as S

from systems import configurations, gpu_context, raw_grids32, state_table

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_cycle_with_host_or_device_arrays_repeats_the_separate_calls():
    from paper_1507_03703_gb300.sampler import Leg, ReplicaExchange
    sys_ = S.config_small(1)
    g32 = raw_grids32(sys_)
    T, alpha, dt = state_table(sys_)
    ctx = gpu_context(sys_, g32, T, alpha, dt)
    bc, cd = sys_.legs
    legs = [(bc.K, 0), (cd.K, bc.K)]
    C, n_cyc, steps, seed = 5, 6, 12, 77
    R = C * (bc.K + cd.K)
    x0 = configurations(sys_, R, seed=81)
    ref = ReplicaExchange(ctx, [Leg(K, o) for K, o in legs], C, x0, seed=seed)
    ukn_ref = []
    for cyc in range(n_cyc):
        ref.hmc(cyc, steps)
        ref.exchange(cyc)
        parts = []
        for li, (K, off) in enumerate(legs):
            u = torch.empty((K, C * K), dtype=torch.float64, device="cuda")
            ctx.reduced_energies(C * K, comps=ref.comps[ref.leg_slice(li)], k_begin=off, k_count=K, u_kn=u)
            parts.append(u.reshape(-1))
        ukn_ref.append(torch.cat(parts).cpu().numpy())
    n_ukn = sum(K * C * K for K, _ in legs)
    # device first, so that the host passes grow the staging buffer after the snapshot's side stream
    # and events exist, and a device pass after them still uses them.  Pinned host arrays are used
    # in place on a device with a coherent host link (staged otherwise); pageable ones are staged.
    for where in ("device", "host", "pageable", "device"):
        st0 = np.concatenate([np.tile(off + np.arange(K), C) for K, off in legs]).astype(np.int32)
        cfg0 = np.concatenate([np.tile(np.arange(K), C) for K, _ in legs]).astype(np.int32)
        arrays = {"x": torch.from_numpy(x0.copy()), "comps": torch.zeros((R, 4), dtype=torch.float64),
                  "state_of": torch.from_numpy(st0), "config_of": torch.from_numpy(cfg0),
                  "counters": torch.zeros(4, dtype=torch.int64), "u_kn": torch.zeros(n_ukn, dtype=torch.float64)}
        if where == "host":
            arrays = {k: v.pin_memory() for k, v in arrays.items()}
        elif where == "pageable":
            arrays = {k: v.numpy() for k, v in arrays.items()}
        else:
            arrays = {k: v.cuda() for k, v in arrays.items()}
        for cyc in range(n_cyc):
            ctx.cycle(legs, C, cyc, arrays["x"], arrays["comps"], arrays["state_of"], arrays["config_of"],
                      n_steps=steps, seed=seed, counters=arrays["counters"], u_kn=arrays["u_kn"])
            u_now = arrays["u_kn"] if where == "pageable" else arrays["u_kn"].cpu().numpy()
            assert np.array_equal(u_now, ukn_ref[cyc]), (where, cyc)
        torch.cuda.synchronize()
        if where == "pageable":
            arrays = {k: torch.from_numpy(v) for k, v in arrays.items()}
        assert torch.equal(arrays["x"].cpu(), ref.x.cpu()), where
        assert torch.equal(arrays["comps"].cpu(), ref.comps.cpu()), where
        assert torch.equal(arrays["state_of"].cpu(), ref.state_of.cpu()), where
        assert torch.equal(arrays["config_of"].cpu(), torch.cat(ref.config_of).cpu()), where
        assert torch.equal(arrays["counters"].cpu()[:3], ref.counters.cpu()[:3]), where
