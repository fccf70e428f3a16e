"""GB300-native batched direct-form IIR filters with closed-form gradients.

Public API (the CUDA library is loaded on first use, never at import):
    paper_2511_14390_gb300.dfilt      -- C-ABI binding + torch.autograd.Function
    paper_2511_14390_gb300.inputs     -- seeded synthetic workloads
"""
__all__ = ["dfilt", "inputs"]


def __getattr__(name):
    if name in ("dfilt", "inputs"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
