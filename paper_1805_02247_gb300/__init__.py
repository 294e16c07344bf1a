"""GB300-native (sm_103a) reconstruction hot path of Modi, Feng & Seljak (2018).

``pmrecon`` binds the C ABI of ``libpmrecon.so`` (include/pmrecon.h);
``synth`` draws the seeded synthetic inputs; ``build`` compiles the library.
"""
