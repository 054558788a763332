"""Helpers shared by the GPU parity tests: oracle keys / ciphertexts and GPU contexts."""
import numpy as np

from oracle import bfv, encoder, ffconv, params


def need_gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def make_ctx(prm):
    from paper_2102_03494_gb300 import he
    need_gpu()
    ctx = he.Context(log_n=prm.log_n, n_q=prm.n_q, n_p=prm.n_p, alpha=prm.alpha, t=prm.t,
                     q_bits=prm.q_bits, p_bits=prm.p_bits)
    assert ctx.he_get_moduli() == prm.q + prm.p + [prm.t]
    return ctx


def oracle_keys(prm, s, steps, seed=2):
    keys, blob = {}, []
    for st in steps:
        g = bfv.galois_of(st, prm.n)
        if g not in keys:
            keys[g] = bfv.galois_key(prm, s, g, seed)
        blob.append(keys[g].reshape(-1))
    return keys, (np.concatenate(blob) if blob else np.zeros(0, dtype=np.uint64))


def gpu_steps(steps):
    from paper_2102_03494_gb300 import he
    return [he.HE_ROW_SWAP if s == bfv.ROW_SWAP else int(s) for s in steps]


def upload_ntt(ctx, ct: bfv.Ct):
    d = ctx.from_numpy(ct.stack())
    ctx.he_to_ntt(d)
    return d


def download_coeff(ctx, d):
    x = d.clone()
    ctx.he_to_coeff(x)
    return ctx.to_numpy(x)


def encrypt_slots(prm, s, v, seed):
    return bfv.encrypt(prm, s, encoder.encode(v, prm), seed)
