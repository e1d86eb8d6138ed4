"""Hyperparameter presets of the Allegro-style potential (configuration only).

Widths follow Table 1 of Allegro-FM (arXiv 2502.06073) for FM64/FM256/FM512, and the two
synthetic-test models: a small l<=1 model (96-atom cubic system) and the l<=2,
3-layer, 32-channel model used for the water / C-S-H / SiO2 / molecule workloads.
avg_num_neighbors (nu) is the normalisation of the environment sum; it is a model
hyperparameter, set per workload to 4/3*pi*rc^3*n rounded.
"""

SMALL = dict(rc=5.0, skin=0.0, n_basis=8, poly_p=6, lmax=1, parity=1, n_layers=2,
             channels=16, two_body=[32, 32], latent=[32, 32], edge_eng=[32],
             avg_num_neighbors=50.0)

FM_WATER = dict(rc=6.0, skin=1.0, n_basis=8, poly_p=6, lmax=2, parity=1, n_layers=3,
                channels=32, two_body=[64, 128, 256], latent=[256], edge_eng=[128],
                avg_num_neighbors=91.0)

FM64 = dict(rc=5.2, skin=1.0, n_basis=8, poly_p=6, lmax=2, parity=1, n_layers=2,
            channels=16, two_body=[16, 32, 64], latent=[64, 64, 64], edge_eng=[64],
            avg_num_neighbors=60.0)
FM256 = dict(FM64, channels=64, two_body=[64, 128, 256], latent=[256, 256, 256],
             edge_eng=[128])
FM512 = dict(FM64, channels=128, two_body=[128, 256, 512], latent=[512, 512, 512],
             edge_eng=[128])

PRESETS = {"small": SMALL, "fm_water": FM_WATER, "fm64": FM64, "fm256": FM256,
           "fm512": FM512}

# nu per workload: 4/3*pi*rc^3*n rounded for the bulk systems (rc = 6 A unless the preset
# says otherwise); for the isolated molecules the batch mean of neighbours within 6 A
NU = {"cubic96": 50.0, "water12288": 91.0, "water4095": 91.0, "csh131072": 82.0,
      "csh512": 82.0, "sio2_4194304": 60.0, "sio2_4096": 60.0, "molecules1024": 33.0,
      "csh_np6326": 60.0}


def preset(name, **over):
    hp = dict(PRESETS[name])
    hp["two_body"] = list(hp["two_body"])
    hp["latent"] = list(hp["latent"])
    hp["edge_eng"] = list(hp["edge_eng"])
    hp.update(over)
    return hp
