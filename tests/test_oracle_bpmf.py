"""Oracle pin for the whole estimator chain ("Estimation": beta_T B = f_BC,L + f'_CD by MBAR over
replica-exchange HMC samples): for a one-atom ligand the BPMF has a closed quadrature,

    B = -kT ln [ int exp(-beta_T (Psi_g(r) + U_I(r))) d^3r / int exp(-beta_T U_I(r)) d^3r ],

with the numerator summed on a sub-lattice of the receptor grid (scipy's trilinear interpolator,
an implementation independent of the oracle's) and the denominator in closed form."""
import numpy as np
import oracle
from paper_1507_03703_gb300 import synthetic as S

from systems import quadrature_bpmf


def test_one_atom_bpmf_matches_quadrature():
    sys_ = S.config_small(1)
    g = sys_.grid
    lig = S.one_atom_ligand()
    ljr, lja, elec = oracle.grid_direct_sum(sys_.receptor, g)
    target = quadrature_bpmf(g, ljr, lja, elec, lig)
    C, K, ncyc, nsteps, dt = 64, 8, 400, 40, 4.0
    rng = np.random.default_rng(5)
    legs = [S.bc_ladder(K, dt_fs=dt), S.cd_ladder(K, dt_fs=dt)]
    f_groups = []
    for li, leg in enumerate(legs):
        osys = oracle.OracleSystem(g, ljr, lja, elec, lig, leg.T, leg.alpha, leg.dt_fs)
        v = rng.normal(size=(C * K, 3))
        v /= np.linalg.norm(v, axis=1)[:, None]
        x0 = (v * 6.0 * rng.uniform(0, 1, size=(C * K, 1)) ** (1 / 3))[:, None, :] + g.center
        comps, st, hacc, _, _ = oracle.run_ladder(osys, x0, C, ncyc, nsteps, seed=21 + li,
                                                  rep_offset=li * C * K, ladder_offset=li * C, burn_in=50)
        # samples are recorded per cycle as C*K slots; group chains into 8 blocks for an error bar
        S_ = comps.shape[0] // (C * K)
        chain = np.tile(np.repeat(np.arange(C), K), S_)
        fl = []
        for grp in range(8):
            m = (chain % 8) == grp
            f, it = oracle.ladder_free_energies(leg.T, leg.alpha, comps[m], st[m])
            assert it > 0
            fl.append(f[-1] - f[0])
        f_all, _ = oracle.ladder_free_energies(leg.T, leg.alpha, comps, st)
        f_groups.append((f_all[-1] - f_all[0], np.array(fl)))
    B = f_groups[0][0] + f_groups[1][0]
    per_group = f_groups[0][1] + f_groups[1][1]
    se = per_group.std(ddof=1) / np.sqrt(len(per_group))
    print("one-atom BPMF", B, "quadrature", target, "se", se)
    assert abs(B - target) < max(0.05, 4 * se), (B, target, se)
