"""Writes tests/golden/data_<workload>.txt: the observed data of the synthetic
workloads.  It calls only the CPU oracle (and the seeded input generators):
R_true = oracle smeared model of a truth draw (one stack per dataset),
R_obs = R_true x lognormal(0, 0.05) noise, e = 0.05 R_true (the Gaussian
likelihood with count-derived standard deviations of Sec. 2.1).

Run:  python tests/golden/make_data.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2509_06924_gb300 import workloads as W  # noqa: E402


def main():
    for name in ("film_1l", "thick_oxide", "oled_cofit", "vi_step"):
        wl = W.make_workload(name, n_stacks=1, data="none")
        n_layers, stacks = W.truth_stacks(name)
        rng = W.noise_rng(name)
        r_obs = np.zeros_like(wl.q)
        r_err = np.zeros_like(wl.q)
        for dsi in range(wl.n_datasets):
            a, b = int(wl.q_off[dsi]), int(wl.q_off[dsi + 1])
            m = oracle.model(n_layers[dsi], stacks[dsi], wl.q[a:b].astype(np.float64),
                             wl.dq[a:b].astype(np.float64), wl.n_quad)
            noise = np.exp(rng.normal(0.0, 0.05, b - a))
            r_obs[a:b] = (m * noise).astype(np.float32)
            r_err[a:b] = (0.05 * m).astype(np.float32)
        header = (f"workload {name}: observed data written by tests/golden/make_data.py from the CPU oracle\n"
                  f"truth draw: workloads.truth_stacks('{name}'); noise lognormal(0, 0.05); e = 0.05 R_true\n"
                  f"quadrature nodes K = {wl.n_quad}")
        path = W.write_data_file(name, wl.q_off, wl.q, wl.dq, r_obs, r_err, header)
        print("wrote", path, int(wl.q_off[-1]), "points")


if __name__ == "__main__":
    main()
