"""Tracker options: physical inputs and every cut of the reconstruction.

The paper (Sec. 2, Sec. 3) describes the cuts qualitatively and prints no
values; the defaults below are this library's readings of it:

* shared-cluster fraction 10 % (Sec. 2 default; 20 % is the loose setting of
  the mitigation described in Sec. 2);
* the "inner region" where Phase II re-attaches clusters = the 20 innermost
  pad rows (Sec. 2 and Sec. 4 both single out rows below 20);
* Phase II candidate depth (tracks may fall back to their k-th candidate) = 4;
* Phase III (Sec. 3): tracks are extrapolated over at most ``ext_rows`` rows
  below their innermost and above their outermost cluster, into the
  neighbouring sector where they leave theirs, with a candidate cut of chi2 < 9
  (stricter than the interpolation cut of 25); off by default, as the paper
  describes it as work in progress;
* seeding iterations on leftover clusters (Sec. 3): ``seed_iters`` sector-
  tracking passes with the same cuts, each later one on the clusters that no
  accepted tracklet of the earlier ones kept; off by default for the same
  reason.
"""
from __future__ import annotations

from dataclasses import asdict, dataclass, field

MODE_STRICT = 0  # FP32, no FMA contraction: bit-identical to the strict CPU oracle
MODE_FAST = 1    # FP32 with FMA contraction


@dataclass
class TrackerOptions:
    bz: float = 0.5                 # tesla
    sigma_y: float = 0.1            # cluster resolution [cm]
    sigma_z: float = 0.1
    ms_theta: float = 1e-3          # scattering angle per pad row [rad]
    link_wy: float = 2.5            # CA neighbour window [cm]
    link_wz: float = 2.5
    link_chi2: float = 1.0          # max squared distance of the middle cluster to the d-u line [cm^2]
    seed_c: tuple = (1.0, 1.0, 0.25, 0.25, 100.0)  # seed covariance diagonal
    follow_chi2: float = 9.0        # cluster pick-up cut during following (2 dof)
    max_snp: float = 0.95           # |sin(phi)| limit of seeding and following
    fit_max_snp: float = 0.99       # limit of refits, merging and the final fit
    score_w: float = 2.0            # selector score = n_clusters - score_w * chi2/ndf
    shared_frac: float = 0.10
    merge_chi2: float = 30.0        # 5-dof match at the common x
    merge_dy: float = 3.0
    merge_dz: float = 3.0
    int_chi2: float = 25.0          # interpolation cut / Phase II candidate cut (2 dof)
    final_chi2: float = 16.0        # simple cut of the last fit iteration
    attach_margin: float = 0.5      # widening of the Phase II search window [cm]
    looper_qpt: float = 1.0 / 0.15  # |q/pT| above which the fit update runs in FP64
    edge_margin: float = 1.0        # following stops beyond the sector edge + this [cm]
    ext_rows: int = 0               # Phase III: rows searched below a track's innermost and
                                    # above its outermost cluster (0: off, <= 32)
    ext_chi2: float = 9.0           # Phase III candidate cut (2 dof), stricter than int_chi2
    seed_iters: int = 1             # sector-tracking iterations; each later one seeds again on
                                    # the clusters the accepted tracklets left (1: off, <= 4)
    # online cluster removal (Sec. 4), run by Tracker.cluster_removal after a tracking call
    cr_mode: int = 0                # 0: off, 1: protective / removal tubes + seeding
                                    # history, 2: also protection 2 (dynamic tube sizes)
    cr_qpt: float = 10.0            # |q/pT| above which a track is very low pT (pT < 0.1 GeV)
    cr_protect: float = 1.5         # protective tube half-width around physics tracks [cm]
    cr_remove: float = 0.75         # removal tube half-width (protection 1: narrower) [cm]
    cr_edge: float = 2.0            # protection 2: sector-edge band [cm]
    cr_occ_w: float = 2.0           # protection 2: occupancy window half-width [cm]
    cr_occ_max: int = 6             # protection 2: clusters in the window above which it applies
    cr_p2_grow: float = 2.0         # protection 2: factor on the protective tube
    cr_p2_shrink: float = 0.5       # protection 2: factor on the removal tube
    cr_leg_dq: float = 0.1          # looper legs: relative |q/pT| difference
    cr_leg_dtgl: float = 0.05       # looper legs: |tan(lambda_a) + tan(lambda_b)|
    cr_leg_dc: float = 3.0          # looper legs: circle-centre distance [cm]
    ac_merge: int = 0               # 1: merge across the central electrode (A <-> C), with
                                    # the z shift of the far side (2 vd t0) estimated
    edge_rows: int = 0              # edge following (Sec. 2): rows followed into the adjacent
                                    # sector beyond a track end at a sector edge (0: off, <= 32)
    edge_min: int = 3               # clusters a segment found there needs to be kept
    max_miss: int = 10              # consecutive empty rows ending the following
    min_hits: int = 10
    merge_max_gap: int = 20         # rows between merged segments
    inner_rows: int = 20
    cand_k: int = 4
    brute_force: int = 0            # oracle only: scan whole rows
    n_rows: int = 152
    n_sectors: int = 36

    def as_dict(self) -> dict:
        return asdict(self)
