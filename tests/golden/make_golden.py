"""Writes the golden fixtures of tests/golden/ (closed forms and the paper's constants).

Nothing here calls the GPU path or the oracle: the bar values are the continuum
closed form (plane strain in 2D) and the constants are transcribed from the paper
(PeTTO, arXiv 2509.06971) with the section each comes from.
Run:  python tests/golden/make_golden.py
"""
import json
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def bar():
    # Uniaxial bar on symmetry rollers, traction t on x = L, modulus E, Poisson nu.
    t, E, nu, h = 0.7, 2.5, 0.3, 0.5
    x2, y2 = 8 * h, 5 * h                 # far corner of the 8 x 5 grid
    x3, y3, z3 = 5 * h, 3 * h, 4 * h      # far corner of the 5 x 3 x 4 grid
    return {
        "_source": "continuum closed form: sigma_xx = t, other stresses 0 (Sec. 3.2 stress law; "
                   "2D plane strain, reading R2)",
        "2d": {"t": t, "E": E, "nu": nu, "h": h, "far_corner_u": [t * (1 - nu ** 2) * x2 / E,
                                                                   -t * nu * (1 + nu) * y2 / E]},
        "3d": {"t": t, "E": E, "nu": nu, "h": h, "far_corner_u": [t * x3 / E, -nu * t * y3 / E,
                                                                   -nu * t * z3 / E]},
    }


def paper_constants():
    return {
        "_source": "PeTTO (arXiv 2509.06971), Sec. 3.1 (heat), Sec. 3.2 (MBB), Sec. 3.3 (3D cantilever)",
        "heat2d": {"dt1_over_dx2": 0.25, "dt2_over_dx": 0.5, "dt3_over_dx4": 500.0, "gamma": 3e-5,
                   "alpha_h": 0.1, "alpha_v": 1e5, "alpha_1": 1e4, "penal": 3.0, "f": 0.01,
                   "kappa_s": 1.0, "kappa_v": 1e-6, "V_s": 0.3, "grid": [512, 512],
                   "apt_sweeps": 500, "pt_sweeps": 500, "loops": 5000, "seconds_gpu": 51, "seconds_cpu": 2173,
                   "_cite": "Sec. 3.1"},
        "mbb": {"theta": 1.0, "dt1_over_dx2": 0.25, "dt2_over_dx": 0.5, "dt3_over_dx4": 500.0,
                "alpha_v": 1e4, "alpha_1": 1e3, "nu": 0.3, "E": [1.0, 0.775, 0.55, 0.325, 0.1],
                "E_void": 1e-6, "V_i": 0.08, "grid": [513, 128], "dofs": 525312,
                "apt_sweeps": 20, "pt_sweeps": 20, "seconds_gpu": 176, "seconds_cpu": 8774,
                "_cite": "Sec. 3.2"},
        "cantilever3d": {"dt1_over_dx2": 1.0 / 6.0, "dt2_over_dx": 0.5, "dt3_over_dx4": 500.0,
                         "E": [1.0, 0.6, 0.2], "E_void": 1e-6, "V_i": 0.1, "grid": [256, 17, 85],
                         "apt_sweeps": 100, "pt_sweeps": 100, "loops": 4000, "seconds_gpu": 796,
                         "seconds_cpu": 36800, "_cite": "Sec. 3.3"},
    }


if __name__ == "__main__":
    for name, obj in (("uniaxial_bar.json", bar()), ("paper_constants.json", paper_constants())):
        with open(os.path.join(HERE, name), "w") as f:
            json.dump(obj, f, indent=1, sort_keys=True)
            f.write("\n")
