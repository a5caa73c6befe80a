"""Analytic profitability model of CREDIT (Sec. III-D), in plain Python.

TEST INFRASTRUCTURE ONLY: the product's model lives in the CUDA library
(`credit_model_eval`); this restatement exists to check it.  Each function is
one equation of the paper, in its notation (Table III):

  Eq. 3  S_CTA(N, P) = ceil(N/P) b_keep + S_scratch <= S_max
  Eq. 4  D_base = D_fixed + N b_reread,  D_cluster = D_fixed
  Eq. 6  D_DSM^w = s P (P-1) sum_l q_l,  D_DSM^r = 0,  K = 2 L
  Eq. 7  B_eff = M N b_B / T_B,  T_save = M N b_reread / B_eff = T_B b_reread / b_B
  Eq. 8  W = ceil(M / clusters),  T_replay = W ceil(N/P) b_keep / (f B_SMEM^r),
         T_DSM = s W (P-1) sum q / (f B_DSM^w(P))
         (the paper's floor(S/P) concurrent clusters is passed in as
         `clusters`, the occupancy the hardware reports)
  (Sec. III-D)  T_deposit = [T_SMEM^w - T_input]^+
  Eq. 9  dT = T_save - T_ctrl - T_replay - T_deposit - T_DSM

The Table IV ablation ("peak bandwidth + serialized staging") replaces B_eff
by the device peak in T_save and charges the whole deposit.
Units: times in us, f in MHz, rates in bytes per cycle, bandwidths in GB/s.
"""
from __future__ import annotations

import math


def capacity_ok(N: int, P: int, b_keep: float, S_scratch: float, S_max: float) -> bool:
    """Eq. 3."""
    return math.ceil(N / P) * b_keep + S_scratch <= S_max


def hbm_traffic(D_fixed: float, N: int, b_reread: float):
    """Eq. 4: (D_base, D_cluster) bytes per row."""
    return D_fixed + N * b_reread, D_fixed


def dsmem_protocol(s: float, P: int, q: list):
    """Eq. 6: (remote write bytes per row, remote read bytes, barriers)."""
    return s * P * (P - 1) * sum(q), 0.0, 2 * len(q)


def effective_bandwidth_gbs(M: float, N: float, b_B: float, T_B_us: float) -> float:
    """Eq. 7, first line (GB/s)."""
    return M * N * b_B / T_B_us / 1e3


def t_save_us(T_B_us: float, b_reread: float, b_B: float) -> float:
    """Eq. 7, second line."""
    return T_B_us * b_reread / b_B


def waves(M: float, clusters: float) -> float:
    """Eq. 8, W."""
    return math.ceil(M / clusters)


def t_replay_us(W: float, N: float, P: float, b_keep: float, f_mhz: float, B_smem_r: float) -> float:
    """Eq. 8, T_replay."""
    return W * math.ceil(N / P) * b_keep / (f_mhz * B_smem_r)


def t_dsm_us(s: float, W: float, P: float, q_sum: float, f_mhz: float, B_dsm_w: float) -> float:
    """Eq. 8, T_DSM (not multiplied by P: the P sources store concurrently)."""
    return s * W * (P - 1) * q_sum / (f_mhz * B_dsm_w)


def t_deposit_us(T_smem_w_us: float, T_input_us: float) -> float:
    """Sec. III-D: only the part of the deposit the input stream does not hide."""
    return max(0.0, T_smem_w_us - T_input_us)


def evaluate(inp: dict, ablation: bool = False) -> dict:
    """All terms of Eq. 7-9 for one (M, N, P); field names as credit_model_eval."""
    M, N, P = inp["M"], inp["N"], inp["P"]
    W = waves(M, max(1.0, inp["active_clusters"]))
    B_eff = effective_bandwidth_gbs(M, N, inp["b_B"], inp["T_B_us"])
    replay = t_replay_us(W, N, P, inp["b_keep"], inp["f_mhz"], inp["B_smem_read"])
    dsm = t_dsm_us(inp["s_bytes"], W, P, inp["q_sum"], inp["f_mhz"], inp["B_dsm_store"])
    smem_w = W * math.ceil(N / P) * inp["b_keep"] / (inp["f_mhz"] * inp["B_smem_store"])
    if ablation:
        save = M * N * inp["b_reread"] / (inp["B_peak_gbs"] * 1e3)
        t_in = 0.0
        deposit = smem_w
    else:
        save = t_save_us(inp["T_B_us"], inp["b_reread"], inp["b_B"])
        t_in = M * N * inp["b_in"] / (B_eff * 1e3)
        deposit = t_deposit_us(smem_w, t_in)
    dT = save - inp["T_ctrl_us"] - replay - deposit - dsm
    return {"W": W, "B_eff_gbs": B_eff, "T_save_us": save, "T_replay_us": replay, "T_dsm_us": dsm,
            "T_deposit_us": deposit, "T_smem_w_us": smem_w, "T_input_us": t_in, "dT_us": dT}


def pick(dts: dict):
    """Sec. III-D selection: the legal P with the largest dT if it is positive,
    else None (keep the non-DSMEM baseline)."""
    best = None
    for P, dT in sorted(dts.items()):
        if dT > 0 and (best is None or dT > dts[best]):
            best = P
    return best


def crossover(widths: list, legal_dts: dict):
    """N*: the smallest tested width with a legal P of positive dT
    (legal_dts[N] = {P: dT} for the legal P only)."""
    for N in sorted(widths):
        if any(v > 0 for v in legal_dts.get(N, {}).values()):
            return N
    return None
