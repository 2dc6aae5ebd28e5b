__kernel void skip_rest(__global int *a, uint n)
{
    uint var0;
    uint var1;
    uint var2;
    uint var3;
    uint var4;
    uint var5;
    var0 = 0u;
    var1 = 0u;
    do {
        var2 = (var0 + 3u);
        if (!(var1 == n)) {
            var3 = (var2 + 5u);
            var4 = var3;
        } else {
            var4 = var2;
        }
        var5 = (var1 + 1u);
        var0 = var4;
        var1 = var5;
    } while (var5 < 4u);
    a[get_local_id(0)] = (int)var4;
}
