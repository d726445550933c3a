"""GB300-native stochastic Hessian / HVP / gradient estimation for a
Gaussian-smoothed rendering loss (Wang, Fischer, Ritschel, "Stochastic
Gradient Estimation for Higher-order Differentiable Rendering").

The compute path is the CUDA library ``libhr`` (C ABI, ``include/hr.h``);
``paper_2412_03489_gb300.hr`` is its thin ctypes binding.
"""
