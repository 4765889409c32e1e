"""Batched unbinned likelihoods on one GB300 (arXiv:2003.12861, Sec. 4).

A model is a computation graph of observables, parameters and PDFs
(Sec. 1); the library evaluates -sum_i log p_i and its gradient over every
event of a dataset in one fused pass on the GPU, fits by BFGS, generates
toys and fits thousands of them at once.  Everything runs in the CUDA
library ``librfgpu.so`` behind the C ABI of ``include/rf.h``; ``api`` only
marshals arguments.  Build it first, from the repository root (the
package is used in place, with the root on ``sys.path``):
``python -m paper_2003_12861_gb300.build``.

Example: f * Gauss(x; mu, sigma) + (1 - f) * (1 + a1 x) on x in [0, 10];
the free parameters, in node order, are theta = (mu, sigma, a1, f)::

    import numpy as np
    from paper_2003_12861_gb300 import api
    from paper_2003_12861_gb300.workloads import Node

    nodes = [Node("obs", (), 0.0, 0.0, 10.0),            # 0: x and its range
             Node("param", (), 5.0, 0.0, 10.0, True),    # 1: mu (start, bounds, free)
             Node("param", (), 1.0, 0.01, 10.0, True),   # 2: sigma
             Node("gauss", (0, 1, 2)),                   # 3: observable, then parameters
             Node("param", (), 0.1, -0.1, 1.0, True),    # 4: a1
             Node("poly", (0, 4)),                       # 5
             Node("param", (), 0.5, 0.0, 1.0, True),     # 6: f
             Node("sum", (3, 5, 6))]                     # 7: PDFs, then fractions
    model = api.Model(nodes, root=7)
    data = api.Data.upload(model, [x])                   # x: float64 array of events
    nll, grad = api.nll_grad(model, data, [5.0, 1.0, 0.1, 0.5])
    r = api.fit(model, data)                             # r["theta"], r["nll"], r["cov"], r["status"]

Several datasets (toys) go in one Data with ``offsets``; ``api.fit`` then
fits all of them in one batched call.  ``api.generate_toys`` draws them on
the device, ``api.RfNLL`` is the torch autograd face of the pass, and
``workloads`` holds the benchmark models (``decay_model``, ``prod3_model``).
"""
